"""Writes explog_tables.h: the breakpoint tables of the table-driven exp and
log (explog.cuh for double, explog_df.cuh for double-float), computed with
mpmath at 200 bits: each entry as the double nearest the exact value, and as
a float pair hi + lo (hi the float nearest the value, lo the float nearest the
remainder, together within 2^-48 relative).

  t2[j]   = 2^(j/64),                          j = 0..63
  logF[j] = log(F_j), or log(F_j / 2) from j = 64,  F_j = 1 + j/128, j = 0..128
  rcpF[j] = 1/F_j

Run: python gen_explog_tables.py  (rewrites explog_tables.h beside it)
"""
import os

import mpmath as mp

mp.mp.prec = 200
EXP_N, LOG_N, LOG_HALF = 64, 129, 64


def _hex(v):
    return float(v).hex()


def _f32(v):
    """The float nearest the mpf v, as a C literal."""
    import numpy as np
    h = np.float32(v)  # via double: exact for these values' float neighbours
    if abs(mp.mpf(float(np.nextafter(h, np.float32(np.inf)))) - v) < abs(mp.mpf(float(h)) - v):
        h = np.nextafter(h, np.float32(np.inf))
    elif abs(mp.mpf(float(np.nextafter(h, np.float32(-np.inf)))) - v) < abs(mp.mpf(float(h)) - v):
        h = np.nextafter(h, np.float32(-np.inf))
    return h


def _pair(v):
    h = _f32(v)
    lo = _f32(v - mp.mpf(float(h)))
    return "{%sf, %sf}" % (float(h).hex(), float(lo).hex())


def tables():
    t2 = [mp.power(2, mp.mpf(j) / EXP_N) for j in range(EXP_N)]
    logF, rcpF = [], []
    for j in range(LOG_N):
        F = 1 + mp.mpf(j) / 128
        logF.append(mp.log(F / 2) if j >= LOG_HALF else mp.log(F))
        rcpF.append(1 / F)
    return t2, logF, rcpF


def render():
    t2, logF, rcpF = tables()
    out = ["// Generated by gen_explog_tables.py: doubles nearest 2^(j/64), log F_j",
           "// (log(F_j / 2) from j = 64) and 1/F_j, F_j = 1 + j/128. Do not edit.",
           "#pragma once", "", "#define OSIRIS_EXPLOG_T2 \\"]
    out += ["  %s, \\" % _hex(v) for v in t2[:-1]] + ["  %s" % _hex(t2[-1]), ""]
    out.append("#define OSIRIS_EXPLOG_LG \\")
    rows = ["  {%s, %s}" % (_hex(a), _hex(b)) for a, b in zip(logF, rcpF)]
    out += [r + ", \\" for r in rows[:-1]] + [rows[-1], ""]
    out.append("#define OSIRIS_EXPLOG_T2_DF \\")
    rows = ["  " + _pair(v) for v in t2]
    out += [r + ", \\" for r in rows[:-1]] + [rows[-1], ""]
    out.append("#define OSIRIS_EXPLOG_LG_DF \\")
    rows = ["  {%s, %s}" % (_pair(a), _pair(b)) for a, b in zip(logF, rcpF)]
    out += [r + ", \\" for r in rows[:-1]] + [rows[-1], ""]
    return "\n".join(out)


if __name__ == "__main__":
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "explog_tables.h")
    with open(path, "w") as fh:
        fh.write(render())
    print("wrote", path)
