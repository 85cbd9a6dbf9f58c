"""Train the learned selector (Section III-H) on GB300 timing labels and write
the tree table the library evaluates.

    python -m paper_2506_20677_gb300.selector.train_trees labels.json ahs_trees.txt

The paper trains an XGBoost classifier on (n, k, H); XGBoost is not available
here, so this uses scikit-learn's gradient-boosted trees on (log2 n, log2 k,
h, key bytes, has payload) -- trees are invariant to monotone transforms of a
feature, so log2 n and log2 k carry the paper's n and k.  Model inputs below
n = 1000 are not used: the library applies the static rules there (Table IV).

Tree table (plain text, whitespace separated):
    ahs-trees 1
    classes C  <C strategy codes>
    features F
    trees T
    nodes M                     (then M lines per tree)
    feature threshold left right v_0 .. v_{C-1}
feature -1 marks a leaf, whose v_c are added to the class scores.  An inner
node sends x to `left` when float32(x[feature]) <= threshold (the rule
scikit-learn's trees apply).  The prediction is the class with the largest
total score, the first one on ties.
"""
from __future__ import annotations

import json
import math
import sys

import numpy as np

MIN_N = 1000


def features_of(row):
    return [math.log2(max(row["n"], 1)), math.log2(row["span"] + 1.0), row["entropy_norm"],
            float(row["key_bytes"]), float(row["payload"])]


STRATEGY_CODE = {"IDENTITY": 1, "SMALL": 2, "COUNTING": 3, "RADIX": 4, "GENERAL": 5}


def load(path):
    with open(path) as fh:
        rows = json.load(fh)["rows"]
    rows = [r for r in rows if r["n"] >= MIN_N]
    X = np.array([features_of(r) for r in rows], dtype=np.float64)
    y = np.array([STRATEGY_CODE[r["label"]] for r in rows], dtype=np.int64)
    return rows, X, y


def fit(X, y, n_estimators=40, max_depth=3, learning_rate=0.2, seed=0):
    from sklearn.ensemble import GradientBoostingClassifier
    m = GradientBoostingClassifier(n_estimators=n_estimators, max_depth=max_depth,
                                   learning_rate=learning_rate, random_state=seed)
    m.fit(X, y)
    return m


def to_table(model) -> str:
    classes = [int(c) for c in model.classes_]
    C = len(classes)
    lr = float(model.learning_rate)
    init = np.asarray(model._raw_predict_init(np.zeros((1, model.n_features_in_)))[0], dtype=np.float64)
    trees = []
    # the initial (prior) scores as a one-leaf tree
    if C == 2:
        init_vec = [0.0, float(init[0])]
    else:
        init_vec = [float(v) for v in init]
    trees.append([(-1, 0.0, 0, 0, init_vec)])
    for stage in model.estimators_:
        for k, est in enumerate(stage):
            t = est.tree_
            nodes = []
            for i in range(t.node_count):
                if t.children_left[i] == -1:
                    v = float(t.value[i].ravel()[0]) * lr
                    vec = [0.0] * C
                    vec[1 if C == 2 else k] = v
                    nodes.append((-1, 0.0, 0, 0, vec))
                else:
                    nodes.append((int(t.feature[i]), float(t.threshold[i]), int(t.children_left[i]),
                                  int(t.children_right[i]), [0.0] * C))
            trees.append(nodes)
    out = ["ahs-trees 1", "classes %d %s" % (C, " ".join(str(c) for c in classes)),
           "features %d" % model.n_features_in_, "trees %d" % len(trees)]
    for nodes in trees:
        out.append("nodes %d" % len(nodes))
        for f, thr, l, r, vec in nodes:
            out.append("%d %.17g %d %d %s" % (f, thr, l, r, " ".join("%.17g" % v for v in vec)))
    return "\n".join(out) + "\n"


def main():
    labels, out = sys.argv[1], sys.argv[2]
    rows, X, y = load(labels)
    from sklearn.ensemble import GradientBoostingClassifier
    from sklearn.model_selection import cross_val_score
    acc = cross_val_score(GradientBoostingClassifier(n_estimators=40, max_depth=3, learning_rate=0.2,
                                                     random_state=0), X, y, cv=5)
    m = fit(X, y)
    with open(out, "w") as fh:
        fh.write(to_table(m))
    counts = {k: int((y == v).sum()) for k, v in STRATEGY_CODE.items()}
    print(json.dumps({"rows": len(rows), "label_counts": counts,
                      "cv5_accuracy_mean": float(acc.mean()), "cv5_accuracy_std": float(acc.std()),
                      "train_accuracy": float(m.score(X, y)), "out": out}))


if __name__ == "__main__":
    main()
