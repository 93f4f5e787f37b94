"""Schedule tuner for the forward calls (pairs, gram, pairs_varlen).

Every schedule the library offers (sigk_opts: rec, rows_per_lane, coef_path)
solves the same explicit scheme of Sec. 3.1; which is fastest depends on the
shape (path lengths, d, dyadic order, batch) and on the GPU.  ``tune`` times
each candidate on the caller's own tensors with CUDA events, checks that the
candidates agree with one another, and keeps the fastest; ``lookup`` returns
the cached choice for a shape, tuning on a miss.  Choices are cached in memory
and in a JSON file (``$SIGK_TUNE_CACHE``, else
``~/.cache/paper_2006_14794_gb300/schedules.json``), keyed by the call, the
shape, the dtype, the GPU name and SM count, and the library version.

Tuning launches kernels and synchronises: do it before a CUDA-graph capture
(``lookup`` refuses to tune while the current stream is capturing).
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, List, Optional, Sequence, Tuple

import torch

from . import sigk
from .sigk import (COEF_FMA, COEF_TC, COEF_TC5, DEFAULT_VARIANT, REC_BAND, REC_CHAIN, REC_PLAIN,
                   REC_STRIP, Schedule, Variant)

_lock = threading.Lock()
_mem: Dict[str, Schedule] = {}

# two candidates agree when their outputs differ by at most this relative error
AGREE_TOL = {torch.float32: 1e-4, torch.float64: 1e-10}
# a candidate whose first run is this many times slower than the best so far
# is not timed further
GIVE_UP_RATIO = 4.0


def cache_path() -> str:
    p = os.environ.get("SIGK_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_2006_14794_gb300",
                        "schedules.json")


def candidates(op: str, dtype: torch.dtype) -> List[Schedule]:
    """Schedules worth timing, roughly fastest-first so that slow ones are cut
    short.  The uneven-length call plans its own stack and band heights on the
    device, so it takes no rows_per_lane; f64 has neither those forms nor the
    tensor-core coefficient kernel."""
    c: List[Schedule] = []
    if op != "pairs_varlen" and dtype == torch.float32:
        c += [Schedule(REC_CHAIN, r, 0) for r in (4, 8, 16)]
        c += [Schedule(REC_BAND, r, 0) for r in (4, 8, 16)]
    if op == "pairs_varlen" and dtype == torch.float32:
        c.append(Schedule(REC_CHAIN, 0, 0))  # warp stacks, coefficients formed in the sweep
        c.append(Schedule(REC_BAND, 0, 0))   # band classes planned on the device
    for orient in (1, 2):   # rows refine the longer / the shorter path
        if dtype == torch.float32:
            for r in (16, 8, 4):
                c.append(Schedule(REC_STRIP, r, COEF_TC5, orient))
                c.append(Schedule(REC_STRIP, r, COEF_FMA, orient))
            c.append(Schedule(REC_STRIP, 16, COEF_TC, orient))
        else:
            c.append(Schedule(REC_STRIP, 8, COEF_FMA, orient))
    c.append(Schedule(REC_PLAIN, 0, 0))
    return c


def shape_key(op: str, tensors: Sequence, scalars: Sequence, device,
              variant: Variant = DEFAULT_VARIANT) -> str:
    """Cache key: call, tensor shapes and dtype, scalar arguments, GPU, library,
    and the scheme / static kernel when they are not the default."""
    props = torch.cuda.get_device_properties(device)
    shapes = ",".join("x".join(str(int(s)) for s in t.shape) for t in tensors)
    dt = str(tensors[0].dtype).replace("torch.", "")
    sc = ",".join(str(int(v)) for v in scalars)
    key = "%s|%s|%s|%s|%s:%d|%s" % (op, dt, shapes, sc, props.name,
                                     props.multi_processor_count, sigk.version())
    vk = variant.key()
    return key + "|" + vk if vk else key


def _load() -> Dict[str, list]:
    try:
        with open(cache_path()) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def _store(key: str, s: Schedule, ms: float) -> None:
    path = cache_path()
    d = _load()
    d[key] = [int(s.rec), int(s.rows_per_lane), int(s.coef_path), int(s.orient), float(ms)]
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".%d.tmp" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def pick(results: Sequence[Tuple[Schedule, Optional[float], Optional[torch.Tensor]]],
         tol: float) -> Tuple[Schedule, float]:
    """The fastest candidate among those that ran (time not None) and agree
    with the first that ran.  A candidate that disagrees is an error of the
    library, not a slower schedule: raise."""
    ref = None
    best: Optional[Tuple[Schedule, float]] = None
    for s, ms, out in results:
        if ms is None:
            continue
        if ref is None:
            ref = (s, out)
        elif out is not None and ref[1] is not None:
            den = ref[1].abs().clamp_min(1e-30)
            err = float(((out - ref[1]).abs() / den).max()) if out.numel() else 0.0
            if not err <= tol:
                raise sigk.SigkError("schedules %s and %s disagree (rel err %.3g)" % (ref[0], s, err))
        if best is None or ms < best[1]:
            best = (s, ms)
    if best is None:
        raise sigk.SigkError("no schedule supports this call")
    return best


def _call(op: str, args, s: Schedule, variant: Variant = DEFAULT_VARIANT):
    if op == "pairs":
        X, Y, lam = args
        return sigk.pairs(X, Y, lam, schedule=s, variant=variant)
    if op == "gram":
        X, Y, lam = args
        return sigk.gram(X, Y, lam, schedule=s, variant=variant)
    if op == "pairs_varlen":
        Xp, xo, Yp, yo, lam, max_len = args
        return sigk.pairs_varlen(Xp, xo, Yp, yo, lam, max_len, schedule=s, variant=variant)
    raise ValueError("no tuner for " + op)


def _time(op, args, s: Schedule, reps: int, best: Optional[float],
          variant: Variant = DEFAULT_VARIANT):
    """(ms per call, output) or (None, None) when the schedule has no instance."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    try:
        e0.record(st)
        out = _call(op, args, s, variant)    # first run: module load, attributes
        e1.record(st)
        torch.cuda.synchronize()
    except sigk.SigkError as e:
        if e.status == sigk.SIGK_EUNSUPPORTED:
            return None, None
        raise
    first = e0.elapsed_time(e1)
    if best is not None and first > GIVE_UP_RATIO * best:
        return first, out
    e0.record(st)
    for _ in range(reps):
        out = _call(op, args, s, variant)
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def tune(op: str, *args, reps: int = 5, store: bool = True,
         variant: Variant = DEFAULT_VARIANT) -> Tuple[Schedule, float]:
    """Times every candidate schedule of ``op`` on these arguments and returns
    (fastest schedule, its ms per call); caches it unless store=False."""
    tensors = [a for a in args if isinstance(a, torch.Tensor)]
    scalars = [a for a in args if not isinstance(a, torch.Tensor)]
    dev = tensors[0].device
    results = []
    best = None
    for s in candidates(op, tensors[0].dtype):
        ms, out = _time(op, args, s, reps, best, variant)
        results.append((s, ms, out))
        if ms is not None and (best is None or ms < best):
            best = ms
    s, ms = pick(results, AGREE_TOL[tensors[0].dtype])
    if store:
        key = shape_key(op, tensors, scalars, dev, variant)
        with _lock:
            _mem[key] = s
            _store(key, s, ms)
    return s, ms


def lookup(op: str, *args, variant: Variant = DEFAULT_VARIANT) -> Schedule:
    """The cached schedule for this call shape; tunes (and caches) on a miss."""
    tensors = [a for a in args if isinstance(a, torch.Tensor)]
    scalars = [a for a in args if not isinstance(a, torch.Tensor)]
    key = shape_key(op, tensors, scalars, tensors[0].device, variant)
    with _lock:
        s = _mem.get(key)
        if s is None:
            v = _load().get(key)
            if isinstance(v, list) and len(v) >= 5:
                s = Schedule(int(v[0]), int(v[1]), int(v[2]), int(v[3]))
                _mem[key] = s
    if s is not None:
        return s
    if torch.cuda.is_current_stream_capturing():
        raise sigk.SigkError("schedule for %s not tuned yet: call it once with schedule='tuned' "
                             "before the capture" % op)
    return tune(op, *args, variant=variant)[0]


def clear_memory_cache() -> None:
    with _lock:
        _mem.clear()
