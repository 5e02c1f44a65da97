"""Autotuner for the library's schedule choices, with a persistent cache.

A choice (the half-bandwidth b of the dense-to-band stage for a route and
size, the number of concurrent workers of the batched solver, the tile
order and digit width of the slice-product kernel) is measured
once per device and problem class: every candidate runs `reps` times after
one untimed run, the median device time wins, and the result is kept in a
JSON cache file so later processes reuse it without measuring.

The cache path is, in order: the `path` argument, the environment variable
FRACLAP_AUTOTUNE_CACHE, or ~/.cache/fraclap_gb300/autotune.json.  A missing
or unreadable cache starts empty; writes go through a temporary file and a
rename, so a crash never leaves a half-written cache.
"""
from __future__ import annotations

import json
import math
import os
import statistics
import time


def default_cache_path() -> str:
    env = os.environ.get("FRACLAP_AUTOTUNE_CACHE")
    if env:
        return env
    return os.path.join(os.path.expanduser("~"), ".cache", "fraclap_gb300", "autotune.json")


def size_bucket(n: int) -> int:
    """Sizes within a factor sqrt(2) share a tuning result: the bucket is
    round(2 log2 n)."""
    return int(round(2.0 * math.log2(max(int(n), 1))))


class Autotuner:
    """Measures candidates once per key and remembers the fastest."""

    def __init__(self, path: str | None = None):
        self.path = path or default_cache_path()
        self.entries = {}
        try:
            with open(self.path) as fh:
                data = json.load(fh)
            if isinstance(data, dict) and isinstance(data.get("entries"), dict):
                self.entries = data["entries"]
        except (OSError, ValueError):
            self.entries = {}

    @staticmethod
    def key(op: str, fields: dict) -> str:
        return op + ":" + json.dumps(fields, sort_keys=True)

    def lookup(self, op: str, fields: dict, candidates):
        e = self.entries.get(self.key(op, fields))
        if e is not None and e.get("best") in list(candidates):
            return e["best"]
        return None

    def choose(self, op: str, fields: dict, candidates, measure, reps: int = 3):
        """The candidate with the smallest median of `reps` calls of
        measure(candidate) (seconds), after one untimed call of each; cached
        under (op, fields) unless the cached winner is no longer a candidate."""
        candidates = list(candidates)
        if not candidates:
            raise ValueError("no candidates")
        hit = self.lookup(op, fields, candidates)
        if hit is not None:
            return hit
        times = {}
        for c in candidates:
            measure(c)  # warm-up: first-use allocations, module loading
            times[c] = statistics.median(measure(c) for _ in range(max(1, reps)))
        best = min(candidates, key=lambda c: (times[c], candidates.index(c)))
        self.entries[self.key(op, fields)] = {
            "best": best, "seconds": {str(c): times[c] for c in candidates}, "reps": reps,
            "when": time.strftime("%Y-%m-%dT%H:%M:%S")}
        self.save()
        return best

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = f"{self.path}.{os.getpid()}.tmp"
        with open(tmp, "w") as fh:
            json.dump({"version": 1, "entries": self.entries}, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


# ----------------------------------------------------------------------------
# the library's tunables (measured on the current CUDA device)
# ----------------------------------------------------------------------------
def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _event_seconds(fn) -> float:
    """Device time of fn() between CUDA events on the current stream."""
    import torch
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3


def best_band_width(n: int, route: str = "mixed", candidates=(32, 64), tuner: Autotuner | None = None,
                    reps: int = 2) -> int:
    """Half-bandwidth b of the dense-to-band stage for an eigendecomposition
    of about n unknowns through `route` ("fp64": eig_full, "mixed":
    eig_full_mixed), measured on the square-grid Laplacian with the nearest
    square number of unknowns (the stage costs depend on n and b, not on
    the shape of the domain)."""
    import torch
    from . import _binding as B
    if route not in ("fp64", "mixed"):
        raise ValueError("route is 'fp64' or 'mixed'")
    tuner = tuner or Autotuner()
    fields = {"device": _device_name(), "route": route, "n_bucket": size_bucket(n)}
    hit = tuner.lookup("eig_band_width", fields, candidates)
    if hit is not None:
        return hit
    m = max(2, int(round(math.sqrt(n))))
    mask = torch.ones((m, m), dtype=torch.uint8, device="cuda")
    h = 1.0 / (m + 1)
    state = {}

    def measure(b):
        if b not in state:
            ctx = B.Context(band_width=int(b))
            state[b] = (ctx, B.fd_assemble(mask, h, ctx=ctx))
        ctx, asm = state[b]
        if route == "mixed":
            return _event_seconds(lambda: B.eig_full_mixed(asm["A"], asm["rowptr"], asm["col"], asm["val"],
                                                           refine_iters=6, ctx=ctx))
        return _event_seconds(lambda: B.eig_full(asm["A"], ctx=ctx))

    return tuner.choose("eig_band_width", fields, candidates, measure, reps)


def best_workers(problems: list, candidates=(4, 8, 16, 32), tuner: Autotuner | None = None,
                 reps: int = 1) -> int:
    """Number of concurrent workers of the batched solver for a list of
    problems in the form fraclap's solve_batched takes, measured on that list
    and cached under its size profile (count, largest and total n, routes)."""
    from . import _binding as B
    tuner = tuner or Autotuner()
    ns = [int(p["A"].shape[0]) for p in problems]
    fields = {"device": _device_name(), "count": len(problems), "n_max_bucket": size_bucket(max(ns or [1])),
              "n_sum_bucket": size_bucket(sum(ns) or 1),
              "mixed": sum(1 for p in problems if p.get("rowptr") is not None)}
    hit = tuner.lookup("batched_workers", fields, candidates)
    if hit is not None:
        return hit
    ctx = B.Context()
    return tuner.choose("batched_workers", fields, candidates,
                        lambda w: _event_seconds(lambda: B.solve_batched(problems, workers=int(w), ctx=ctx)), reps)


def best_ozaki_schedule(n: int, slices: int = 7, groups=(0, 4, 8, 16), bits=(7,), tiles=(128, 192, 256),
                        clusters=(1, 2), tuner: Autotuner | None = None, reps: int = 2,
                        cols: int | None = None) -> dict:
    """Tile order (raster group of tile rows), tile width, cluster size (CTAs
    sharing a B tile by TMA multicast) and digit width of the slice-product
    kernel for the refinement's residual product X^T X of an n x n X with
    `slices` BF16 slices (or, with cols, the apply's product V^T F of an
    n x n V and an n x cols F), measured on seeded matrices of that size
    through fraclap_dgemm_ozaki.  Returns {"ozaki_group": G, "ozaki_bits": w,
    "ozaki_tile_n": t, "ozaki_cluster": c}; apply it with
    apply_schedule(ctx, ...).  The digit widths tried default to 7 alone:
    8-bit digits (28 instead of 36 slice pairs for 7 slices) measured the same
    kernel time on a GB300 at n = 4096 and 8810, their four times more chunk
    sums taking what the pairs save."""
    import torch
    from . import _binding as B
    tuner = tuner or Autotuner()
    cands = [f"{g}/{w}/{t}/{c}" for c in clusters for t in tiles for w in bits for g in groups]
    fields = {"device": _device_name(), "n_bucket": size_bucket(n), "slices": int(slices)}
    if cols is not None:
        fields["cols_bucket"] = size_bucket(cols)
    nc = n if cols is None else int(cols)
    hit = tuner.lookup("ozaki_schedule", fields, cands)
    if hit is None:
        gen = torch.Generator(device="cpu").manual_seed(n)
        X = (torch.randn(n, n, generator=gen, dtype=torch.float64) / n ** 0.5).cuda()
        Y = X if cols is None else (torch.randn(nc, n, generator=gen, dtype=torch.float64) / n ** 0.5).cuda().t()
        C = torch.empty(nc, n, dtype=torch.float64, device="cuda").t()
        ctx = B.Context()
        ws = torch.empty(ctx.lib.fraclap_dgemm_ozaki_workspace_bytes(n, nc, n, slices), dtype=torch.uint8,
                         device="cuda")

        def measure(c):
            g, w, t, cl = (int(x) for x in c.split("/"))
            ctx.set_schedule("ozaki_group", g)
            ctx.set_schedule("ozaki_bits", w)
            ctx.set_schedule("ozaki_tile_n", t)
            ctx.set_schedule("ozaki_cluster", cl)

            def run():
                import ctypes
                st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
                ctx.check(ctx.lib.fraclap_dgemm_ozaki(ctx.handle, 1, 0, n, nc, n, 1.0, B._ptr(X), n, B._ptr(Y), n,
                                                      0.0, B._ptr(C), n, int(slices), B._ptr(ws), ws.numel(), st))
            return _event_seconds(run)

        hit = tuner.choose("ozaki_schedule", fields, cands, measure, reps)
    g, w, t, cl = (int(x) for x in hit.split("/"))
    return {"ozaki_group": g, "ozaki_bits": w, "ozaki_tile_n": t, "ozaki_cluster": cl}


def apply_schedule(ctx, schedule: dict) -> None:
    """Sets every knob of `schedule` ({knob: value}) on a binding Context."""
    for knob, value in schedule.items():
        ctx.set_schedule(knob, value)
