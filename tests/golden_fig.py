"""Parser for tests/golden/figure1_figure2.txt (the paper's running example)."""
import os

import numpy as np

from paper_2206_10435_gb300.datagen import Query, Relation

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "figure1_figure2.txt")
ATTR = {"A": 0, "B": 1, "C": 2, "D": 3}


def load():
    tables, result, gfjs, facts = {}, [], {}, []
    cur = None
    with open(PATH) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            w = line.split()
            if w[0] == "table":
                cur = (w[1], w[2:], [])
                tables[w[1]] = cur
            elif w[0] == "result":
                first, last = int(w[1]), int(w[2])
                result.extend([tuple(int(x) for x in w[3:])] * (last - first + 1))
                cur = None
            elif w[0] == "gfjs":
                gfjs[w[1]] = [tuple(int(x) for x in p.split(":")) for p in w[2:]]
            elif w[0] in ("uir", "repeat"):
                facts.append(w)
            else:
                cur[2].append([int(x) for x in w])
    rels = []
    for name in ("T1", "T2", "T3"):
        _, cols, rows = tables[name]
        arr = np.array(rows, dtype=np.int32)
        rels.append(Relation(name, [ATTR[c] for c in cols],
                             [arr[:, i].copy() for i in range(arr.shape[1])], []))
    q = Query("figure1", rels, {v: k for k, v in ATTR.items()})
    return q, result, gfjs, facts
