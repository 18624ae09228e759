"""Readers for the hand-derived fixtures under tests/golden/."""
import os

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def num(tok: str) -> float:
    t = tok.strip()
    if t.lstrip("+-").startswith("0x"):
        return float.fromhex(t)
    return float(t)


def _lines(name):
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line


def fixed_cases():
    for line in _lines("find_bin_fixed.txt"):
        nb, a, b, x, exp = line.split()
        yield int(nb), num(a), num(b), num(x), int(exp)


def variable_cases():
    for line in _lines("find_bin_variable.txt"):
        e, x, exp = line.split()
        yield [num(t) for t in e.split(",")], num(x), int(exp)


def fill_cases():
    case = None
    for line in _lines("fill_small.txt"):
        head, *rest = line.split()
        if head == "case":
            case = {"name": rest[0], "axes": [], "events": [], "weights": [],
                    "stat_overflows": 0, "bins": {}, "stats": []}
        elif head == "axis":
            if rest[0] == "fixed":
                case["axes"].append({"kind": "fixed", "nbins": int(rest[1]),
                                     "xmin": num(rest[2]), "xmax": num(rest[3])})
            else:
                case["axes"].append({"kind": "variable",
                                     "edges": [num(t) for t in rest[1].split(",")]})
        elif head == "stat_overflows":
            case["stat_overflows"] = int(rest[0])
        elif head == "event":
            i = rest.index("w")
            case["events"].append([num(t) for t in rest[:i]])
            case["weights"].append(num(rest[i + 1]))
        elif head == "bins":
            for kv in rest:
                k, v = kv.split(":")
                case["bins"][int(k)] = num(v)
        elif head == "stats":
            case["stats"] = [num(t) for t in rest]
        elif head == "end":
            yield case
            case = None
