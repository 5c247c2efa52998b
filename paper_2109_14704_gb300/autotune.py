"""Autotuner for the transform kernels.

For a batch shape (N, limbs, count) it times every transform shape the
library built for that degree (he_ntt_shapes: words per CTA, i.e. how many
stages run across the CTAs of a cluster versus inside one CTA's shared
memory; words per thread, i.e. radix-8 or radix-16 register rounds and with
them the threads per CTA; and the CTAs per SM the kernels are compiled for,
i.e. their register budget -- the paper tuned the same knobs by hand:
radix, SLM threshold and register slots, Sec. III-B, Sec. IV-A), each
launched either as one cluster per limb or as a persistent grid walking the
limbs, and keeps the fastest for each direction. Each candidate is first checked once: its
forward output must equal the default shape's output bit for bit and its
inverse must restore the input exactly. Candidates are timed with CUDA
events (forward + inverse, median of `reps` after warm-up); the fastest wins,
ties going to the earlier candidate. Results are cached in a JSON file keyed
by device, N, limbs and count, and applied with he_ntt_set_shape so that the
plain he_ntt_fwd / he_ntt_inv calls use them.

For uneven batches, tune_plan compares the single mixed-degree launch with
per-degree launches (one cluster per limb) in each degree's tuned shape.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import he
from .synth import Rng

DEFAULT_CACHE = os.environ.get(
    "HE_AUTOTUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "paper_2109_14704_gb300", "autotune.json"))


def _load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save_cache(path, cache):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _device_key():
    import torch
    return torch.cuda.get_device_name(torch.cuda.current_device())


def _time(fn, reps, warmup):
    import torch
    s = torch.cuda.current_stream()
    for _ in range(warmup):
        fn()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return statistics.median(times)


def default_moduli(N: int, limbs: int) -> list[int]:
    two_n = 2 * N
    half = (limbs + 1) // 2
    return (he.primes_generate(60, two_n, half) + he.primes_generate(50, two_n, limbs - half))[:limbs]


def tune_uniform(N: int, limbs: int, count: int, moduli=None, reps: int = 10, warmup: int = 3,
                 cache_path: str | None = DEFAULT_CACHE, apply: bool = True, force: bool = False) -> dict:
    """Pick, separately for he_ntt_fwd and he_ntt_inv, the fastest built
    shape (words per CTA, words per thread, one cluster per limb or
    persistent) on `count` polynomials of `limbs` limbs at degree N."""
    import torch

    key = f"{_device_key()}|uniform3|N={N}|limbs={limbs}|count={count}"
    cache = _load_cache(cache_path) if cache_path else {}
    if not force and key in cache:
        res = cache[key]
        if apply:
            _apply(N, res)
        return res

    qs = list(moduli) if moduli is not None else default_moduli(N, limbs)
    tables = he.NttTables(N, qs)
    r = Rng(0xA070)
    x = np.stack([r.uniform_limbs(qs, N) for _ in range(count)])
    x_dev = torch.from_numpy(x.view(np.int64)).cuda()
    d = torch.empty_like(x_dev)
    shapes = he.ntt_shapes(N)

    # reference output: the default shape
    he.ntt_set_shape(N, 0, 0, 0)
    d.copy_(x_dev)
    he.ntt_fwd(d, N, limbs, count, tables)
    ref = d.clone()

    cands = []
    # shape = [log_block, log_thread_words, persistent, ctas_per_sm]
    configs = [(lb, le, pers, occ) for pers in (0, 1) for (lb, le, occ) in shapes]
    try:
        for idx, (lb, le, pers, occ) in enumerate(configs):
            he.ntt_set_shape(N, lb, le, pers, ctas_per_sm=occ)
            d.copy_(x_dev)
            he.ntt_fwd(d, N, limbs, count, tables)
            ok_fwd = bool(torch.equal(d, ref))
            he.ntt_inv(d, N, limbs, count, tables)
            ok_inv = bool(torch.equal(d, x_dev))
            if not (ok_fwd and ok_inv):
                cands.append({"index": idx, "shape": [lb, le, pers, occ], "ok": False})
                continue
            ms_f = _time(lambda: he.ntt_fwd(d, N, limbs, count, tables), reps, warmup)
            ms_i = _time(lambda: he.ntt_inv(d, N, limbs, count, tables), reps, warmup)
            cands.append({"index": idx, "shape": [lb, le, pers, occ], "ok": True, "ms_fwd": ms_f, "ms_inv": ms_i})
    finally:
        he.ntt_set_shape(N, 0, 0, 0)
    good = [c for c in cands if c["ok"]]
    if not good:
        raise RuntimeError(f"no transform shape for N = {N} passed its check")
    bf = min(good, key=lambda c: (c["ms_fwd"], c["index"]))
    bi = min(good, key=lambda c: (c["ms_inv"], c["index"]))
    d0 = next((c for c in good if c["index"] == 0), None)
    res = {"fwd": bf["shape"], "inv": bi["shape"], "ms_fwd": bf["ms_fwd"], "ms_inv": bi["ms_inv"],
           "default_ms_fwd_inv": (d0["ms_fwd"] + d0["ms_inv"]) if d0 else None, "candidates": cands}
    if cache_path:
        cache = _load_cache(cache_path)
        cache[key] = res
        _save_cache(cache_path, cache)
    if apply:
        _apply(N, res)
    return res


def _apply(N, res):
    for direction, key in ((he.FORWARD, "fwd"), (he.INVERSE, "inv")):
        lb, le, pers, occ = (list(res[key]) + [0])[:4]
        he.ntt_set_shape(N, lb, le, pers, direction=direction, ctas_per_sm=occ)


def tune_plan(polys, reps: int = 10, warmup: int = 3, shapes_per_degree: dict | None = None) -> dict:
    """Compare, for an uneven batch given as NttPlan entries (tensor, tables,
    N, limbs, first_prime), the single mixed-degree launch (when every N is
    in [2^12, 2^15]) with per-degree launches in the given (or default)
    shapes. Returns the winning configuration: {"shapes": {...}} to pass to
    NttPlan (an empty dict selects the mixed launch)."""
    import torch

    degrees = sorted({p[2] for p in polys})
    options = []
    if all(4096 <= N <= 32768 for N in degrees):
        options.append({})
    per_degree = {N: tuple((shapes_per_degree or {}).get(N, he.ntt_shapes(N)[0][:2])) for N in degrees}
    options.append(per_degree)
    saved = [p[0].clone() for p in polys]
    results = []
    for idx, shapes in enumerate(options):
        plan = he.NttPlan(polys, shapes=shapes or None)

        def step():
            plan.fwd()
            plan.inv()

        step()
        ok = all(torch.equal(p[0], s) for p, s in zip(polys, saved))
        ms = _time(step, reps, warmup) if ok else None
        results.append({"index": idx, "shapes": {str(k): list(v) for k, v in shapes.items()}, "ok": ok,
                        "ms_fwd_inv": ms, "launches_per_direction": plan.launches})
        plan.close()
    good = [r for r in results if r["ok"]]
    if not good:
        raise RuntimeError("no plan configuration passed its check")
    best = min(good, key=lambda r: (r["ms_fwd_inv"], r["index"]))
    return {"best": best, "candidates": results,
            "shapes": {int(k): tuple(v) for k, v in best["shapes"].items()}}


def tune_mul_relin_rescale(ctx, key, level: int, count: int, reps: int = 10, warmup: int = 3,
                           apply: bool = True) -> dict:
    """Pick the words per thread (radix-8 or radix-16 rounds) of a context's
    key-switching and rescale kernels for `count` MulLinRS at `level`:
    each candidate must reproduce the default's output bit for bit."""
    import torch

    N = ctx.N
    qs = ctx.data_moduli[:level + 1]
    r = Rng(0xA071)
    mk = lambda: torch.from_numpy(np.stack([np.stack([r.uniform_limbs(qs, N) for _ in range(2)])
                                            for _ in range(count)]).view(np.int64)).cuda()
    a, b = mk(), mk()
    out = torch.empty((count, 2, level, N), dtype=torch.int64, device="cuda")
    scratch = torch.empty(ctx.mrr_scratch_bytes(level, count) // 8, dtype=torch.int64, device="cuda")
    ctx.set_eval_shape(0)
    he.mul_relin_rescale(out, a, b, count, key, ctx, level, scratch)
    ref = out.clone()
    cands = []
    for idx, le in enumerate((4, 3)):
        ctx.set_eval_shape(le)
        out.zero_()
        he.mul_relin_rescale(out, a, b, count, key, ctx, level, scratch)
        ok = bool(torch.equal(out, ref))
        ms = _time(lambda: he.mul_relin_rescale(out, a, b, count, key, ctx, level, scratch), reps, warmup) \
            if ok else None
        cands.append({"index": idx, "log_thread_words": le, "ok": ok, "ms": ms})
    good = [c for c in cands if c["ok"]]
    best = min(good, key=lambda c: (c["ms"], c["index"]))
    ctx.set_eval_shape(best["log_thread_words"] if apply else 0)
    return {"log_thread_words": best["log_thread_words"], "candidates": cands}
