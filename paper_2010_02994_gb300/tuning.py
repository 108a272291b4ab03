"""Tile-shape tuning table: measure with the library's autotuner, keep as JSON.

The table maps a GPU name to entries {"d": D, "bucket": ceil(log2 N),
"warps": W, "col_groups": G, "ctas_per_sm": C, "ms": t}: W row groups of
warps (the pair block size), G column groups, at most C persistent CTAs per
SM.  Entries without "col_groups" predate the column groups and are skipped.  `load_into(ctx)` copies the entries
for the context's GPU into the context; `autotune(ctx, t, X, params)` times
every shape on the caller's data, stores the best in the context, and
`save(...)` writes the table.  The timing itself runs in the library
(hawkes_autotune); this module only keeps the file.
"""
from __future__ import annotations

import ctypes
import json
import math
import os

import torch

from . import _lib
from .api import HawkesContext, _dev_f64, _ptr, _shape, params_struct

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def gpu_name(device: int = 0) -> str:
    return torch.cuda.get_device_name(device)


def bucket(n: int) -> int:
    return max(0, math.ceil(math.log2(max(1, n))))


def read(path: str = DEFAULT_PATH) -> dict:
    if not os.path.exists(path):
        return {}
    with open(path) as f:
        return json.load(f)


def load_into(ctx: HawkesContext, path: str = DEFAULT_PATH) -> int:
    """Copy the table's entries for this GPU into the context; returns how many."""
    entries = [e for e in read(path).get(gpu_name(ctx.device), []) if "col_groups" in e]
    for e in entries:
        ctx.check(ctx.lib.hawkes_ctx_set_tuning(ctx.handle, int(e["d"]), int(e["bucket"]), int(e["warps"]),
                                                int(e["col_groups"]), int(e["ctas_per_sm"])))
    return len(entries)


def autotune(ctx: HawkesContext, t, X, params) -> dict:
    """Time every tile shape on (t, X) and keep the fastest in the context."""
    t = _dev_f64(t, "t")
    X = _dev_f64(X, "X")
    n, d, X = _shape(t, X)
    w, wc, c, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
    p = params_struct(params)
    ctx.check(ctx.lib.hawkes_autotune(ctx.handle, _ptr(t), _ptr(X), n, d, ctypes.byref(p), ctx.stream(),
                                      ctypes.byref(w), ctypes.byref(wc), ctypes.byref(c), ctypes.byref(ms)))
    return {"d": d, "bucket": bucket(n), "n": n, "warps": w.value, "col_groups": wc.value, "ctas_per_sm": c.value,
            "ms": ms.value}


def save(entries: list, device: int = 0, path: str = DEFAULT_PATH) -> None:
    """Merge entries into the table under this GPU's name."""
    table = read(path)
    name = gpu_name(device)
    cur = {(e["d"], e["bucket"]): e for e in table.get(name, [])}
    for e in entries:
        cur[(e["d"], e["bucket"])] = e
    table[name] = sorted(cur.values(), key=lambda e: (e["d"], e["bucket"]))
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _random_events(n: int, d: int, seed: int, device):
    """Uniform events: the pair kernels' cost does not depend on the values."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    t = torch.sort(torch.rand(n, generator=g, dtype=torch.float64) * 365.0).values
    X = torch.rand(n, d, generator=g, dtype=torch.float64) * 20.0
    return t.to(device), X.to(device)


def main(argv=None) -> int:
    """Tune every (dimension, size) pair given and merge the results into a table:
        python -m paper_2010_02994_gb300.tuning --d 1 2 4 8 --n 1000 10000 100000 --out tuning.json"""
    import argparse

    ap = argparse.ArgumentParser()
    ap.add_argument("--d", type=int, nargs="+", default=[1, 2, 3, 4, 5, 6, 7, 8])
    ap.add_argument("--n", type=int, nargs="+",
                    default=[600, 1000, 2000, 4000, 8000, 16000, 32000, 64000, 100000])
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--out", default=DEFAULT_PATH)
    args = ap.parse_args(argv)
    params = {"mu0": 0.5, "tau_x": 1.0, "tau_t": 14.0, "theta": 0.5, "omega": 0.5, "h": 0.1}
    ctx = HawkesContext(device=args.device, max_n=max(args.n), max_d=max(args.d), tuning=False)
    entries = []
    dev = torch.device("cuda", args.device)
    for d in args.d:
        for n in args.n:
            t, X = _random_events(n, d, 17 * d + n, dev)
            e = autotune(ctx, t, X, params)
            entries.append(e)
            print(f"d={d} n={n} bucket={e['bucket']}: warps={e['warps']} col_groups={e['col_groups']} "
                  f"ctas/SM={e['ctas_per_sm']} {e['ms']:.4f} ms", flush=True)
    save(entries, args.device, args.out)
    ctx.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
