import os

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name):
    out = {}
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            k, v = line.split("=", 1)
            vals = [float(x) for x in v.split(",")]
            out[k.strip()] = vals if len(vals) > 1 else vals[0]
    return out
