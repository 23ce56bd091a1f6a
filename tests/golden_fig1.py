"""Parser for tests/golden/fig1.txt (the paper's Fig. 1 / Fig. 2 worked example)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    cols, snodes, tree, sizes, update, updates, relind = {}, {}, [], {}, {}, {}, {}
    with open(os.path.join(HERE, "golden", "fig1.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            head, _, rest = line.partition(":")
            vals = rest.split()
            kw = head.split()
            if kw[0] == "col":
                cols[int(kw[1])] = [int(v) for v in vals]
            elif kw[0] == "snode":
                snodes[kw[1]] = [int(v) for v in vals]
            elif kw[0] == "tree":
                tree = [tuple(e.split(">")) for e in vals]
            elif kw[0] == "size":
                sizes[kw[1]] = tuple(int(v) for v in vals)
            elif kw[0] == "update":
                update[kw[1]] = [int(v) for v in vals]
            elif kw[0] == "updates":
                updates[kw[1]] = vals
            elif kw[0] == "relind":
                relind[(kw[1], kw[2])] = [int(v) for v in vals]
    return dict(cols=cols, snodes=snodes, tree=tree, sizes=sizes, update=update,
                updates=updates, relind=relind)
