"""Readers for the text fixtures in this folder (paper data, cited inside)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def psi_table():
    """Returns (orders, orients, psi): orders[k] = (first, second, third) pair
    names, orients[k] = three directed edges as 'xy' strings, psi[k][r] = type
    (1-based k, r, types)."""
    orders, orients, psi = {}, {}, {}
    with open(os.path.join(HERE, "psi_table.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "order":
                orders[int(line[1])] = tuple(line[2:5])
            elif line[0] == "orient":
                orients[int(line[1])] = tuple(line[2:5])
            elif line[0] == "psi":
                psi[int(line[1])] = {r + 1: int(v) for r, v in enumerate(line[2:10])}
    return orders, orients, psi


def hand_cases():
    """Returns a list of (name, edges [(s, d, t)], [(delta triple, expected 8)])."""
    cases = []
    with open(os.path.join(HERE, "hand_cases.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].split()
            if not line:
                continue
            if line[0] == "case":
                cases.append((line[1], [], []))
            elif line[0] == "edge":
                cases[-1][1].append((int(line[1]), int(line[2]), int(line[3])))
            elif line[0] == "delta":
                arrow = line.index("->")
                d = tuple(int(x) for x in line[1:arrow])
                exp = [int(x) for x in line[arrow + 1:]]
                cases[-1][2].append((d, exp))
    return cases


def power_law_counts():
    """The oracle's counts on the full power-law workload, written by
    make_power_law_counts.py.  Returns (fields, [(delta triple, counts[8])]):
    fields holds 'sha256' (of the src, dst, t arrays) and the static
    statistics n, m, m_s, tau, sigma_max, work_bytes, prod as ints."""
    fields, rows = {}, []
    with open(os.path.join(HERE, "power_law_1m_counts.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            key, val = (x.strip() for x in line.split(":", 1))
            if key.startswith("delta "):
                rows.append((tuple(int(x) for x in key.split()[1:]), [int(x) for x in val.split()]))
            elif key == "sha256":
                fields[key] = val
            else:
                fields[key] = int(val)
    return fields, rows
