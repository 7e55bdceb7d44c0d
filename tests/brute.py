"""Independent brute-force restatement of the sampling path, for tiny traces.

Written from the definitions, not from the oracle's streaming loop:

* Section 3.2: after a sample at position p (or the trace start, p = -1, with the
  counter at its entry value c0), the next sample is the first j > p at which
  |c0' + (P_j - P_p)| >= T, where P is the inclusive prefix sum of deltas and c0'
  is c0 for the first window and 0 afterwards.  Found by linear search per window.
* Section 3.3: window totals are plain sums over (p, j]; the footprint is F0 + P_j.
* Section 3.4: high-water crossings are the growth samples whose footprint beats
  every earlier growth-sample footprint and F0; object k is reclaimed if some free
  strictly between crossing k and crossing k+1 carries its address; the last object
  is still open.
* Section 3.5: the number of copy samples at memcpy j is the number of multiples of
  T_c passed by the running byte count, floor((phi+S_j)/T_c) - floor((phi+S_{j-1})/T_c).

Python integers throughout, so nothing overflows.
"""
from __future__ import annotations


def samples(delta, addr, line, py, T, F0=0):
    n = len(delta)
    P = []
    acc = 0
    for d in delta:
        acc += int(d)
        P.append(acc)
    out = []
    p = -1
    while True:
        base = P[p] if p >= 0 else 0
        j = next((j for j in range(p + 1, n) if abs(P[j] - base) >= T), None)
        if j is None:
            break
        win = [int(d) for d in delta[p + 1:j + 1]]
        pys = [int(x) for x in py[p + 1:j + 1]]
        A = sum(d for d in win if d > 0)
        F = sum(-d for d in win if d < 0)
        Apy = sum(d for d, f in zip(win, pys) if d > 0 and f)
        Fpy = sum(-d for d, f in zip(win, pys) if d < 0 and f)
        out.append(dict(idx=j, kind=1 if P[j] - base > 0 else -1, A=A, F=F, A_py=Apy, F_py=Fpy,
                        footprint=F0 + P[j], line=int(line[j]), is_python=int(py[j])))
        p = j
    return out


def hwm_crossings(smp, F0=0):
    best = F0
    hs = []
    for k, s in enumerate(smp):
        s["is_hwm"] = 0
        if s["kind"] > 0 and s["footprint"] > best:
            best = s["footprint"]
            s["is_hwm"] = 1
            hs.append(k)
    return hs


def leak_pairs(delta, addr, smp, n_lines, F0=0):
    hs = hwm_crossings(smp, F0)
    mallocs = [0] * n_lines
    frees = [0] * n_lines
    objs = [(smp[k]["idx"], int(addr[smp[k]["idx"]]), smp[k]["line"]) for k in hs]
    for k, (h, a, l) in enumerate(objs):
        mallocs[l] += 1
        if k + 1 < len(objs):
            h_next = objs[k + 1][0]
            if any(int(delta[i]) < 0 and int(addr[i]) == a for i in range(h + 1, h_next)):
                frees[l] += 1
    return mallocs, frees


def line_stats(smp, n_lines):
    rows = [dict(n_growth=0, n_shrink=0, A=0, F=0, A_py=0, F_py=0, net=0) for _ in range(n_lines)]
    for s in smp:
        r = rows[s["line"]]
        r["n_growth" if s["kind"] > 0 else "n_shrink"] += 1
        for k in ("A", "F", "A_py", "F_py"):
            r[k] += s[k]
        r["net"] += s["A"] - s["F"]
    return rows


def copy_stats(size, line, py, Tc, phi, n_lines):
    samp = [[0, 0] for _ in range(n_lines)]
    byts = [[0, 0] for _ in range(n_lines)]
    S_prev = 0
    for s, l, f in zip(size, line, py):
        S = S_prev + int(s)
        q = (phi + S) // Tc - (phi + S_prev) // Tc
        samp[int(l)][int(f)] += q
        byts[int(l)][int(f)] += q * Tc
        S_prev = S
    return samp, byts
