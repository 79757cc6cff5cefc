"""Launch-shape autotuner for the two blend kernels.

The blend kernels take the number of pixels each thread owns (1, 2 or 4) as a
launch parameter: more pixels per thread share shared-memory reads and warp
reductions, fewer keep more warps resident.  Which wins depends on the scene
(splats per tile, pixels each splat reaches, feature width), so the tuner
times every supported shape on the caller's own frame with CUDA events and
returns raster parameters with the fastest ones.  The rendered images do not
depend on the shape; gradients differ only by the order of float atomics.
"""
from __future__ import annotations

import dataclasses

import torch

from . import _lib as L
from .raster import RasterParams, Renderer

CANDIDATES = (1, 2, 4)
WARP_CANDIDATES = (1, 2)   # one 32-thread block per pixel group (fwd_blocks / bwd_blocks = 1)
BATCH_CANDIDATES = (64, 128, 256)  # splats staged per round by the per-tile forward


def _time(fn, reps: int, stream) -> float:
    fn()                                   # warm-up (and module load)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(reps):
        fn()
    ev[1].record(stream)
    ev[1].synchronize()
    return ev[0].elapsed_time(ev[1]) / reps


_PREFIX = {L.GS_BWD_BLOCKS_GROUP: "w", L.GS_BLOCKS_QUEUE: "q", L.GS_BLOCKS_RING: "r"}
_BLOCKS = {"w": L.GS_BWD_BLOCKS_GROUP, "q": L.GS_BLOCKS_QUEUE, "r": L.GS_BLOCKS_RING}


def shape_keys(p: RasterParams):
    """The (forward, backward) timing keys of the launch shapes of RasterParams p."""
    key = lambda blocks, np_: _PREFIX[blocks] + str(np_) if blocks in _PREFIX else np_
    return key(p.fwd_blocks, p.fwd_px_per_thread), key(p.bwd_blocks, p.bwd_px_per_thread)


def parse_shapes(text: str) -> dict:
    """RasterParams fields for "fwd,bwd" shape keys such as "2,w2", "q2,w2", "r2,w2" or, with
    the forward's staged batch, "2@64,w2"."""
    f_s, b_s = text.split(",")
    f_s, _, batch = f_s.partition("@")
    blocks = lambda k: _BLOCKS.get(k[0], L.GS_BWD_BLOCKS_TILE)
    out = dict(fwd_px_per_thread=int(f_s.lstrip("wqr")), fwd_blocks=blocks(f_s),
               bwd_px_per_thread=int(b_s.lstrip("wqr")), bwd_blocks=blocks(b_s))
    if batch:
        out["fwd_batch"] = int(batch)
    return out


def tune_blend(r: Renderer, field, grad_mode: int = L.GS_GRAD_MAP, reps: int = 5, verbose: bool = False,
               factored: bool = False):
    """Returns (RasterParams with the fastest fwd/bwd launch shapes, timings in ms).  Shapes
    are keyed by pixels per thread (one block per tile), "w1", "w2" (one 32-thread block
    per pixel group) and, for the forward, "q1", "q2", "q4" (resident blocks taking tiles
    from a work counter) and "r2", "r2@64" (the tile's splats staged into a ring of batch
    slots that each warp walks at its own pace); for a per-tile forward the splats it stages
    per round are then timed at 64, 128 and 256 (timings["fwd_batch"]).

    The renderer's image gradients (r.g_*) must hold the gradients to time the
    backward with (e.g. after a loss call; with factored, a factored loss call, and only the
    per-group shapes, which alone take that form, are timed); the projection and binning
    are run here.
    """
    stream = torch.cuda.current_stream()
    base = r.params
    r.project(field)
    r.bin_sort()
    timings = {"fwd": {}, "bwd": {}}
    fshapes = {np_: dict(fwd_px_per_thread=np_, fwd_blocks=L.GS_BWD_BLOCKS_TILE) for np_ in CANDIDATES}
    fshapes.update({f"w{np_}": dict(fwd_px_per_thread=np_, fwd_blocks=L.GS_BWD_BLOCKS_GROUP)
                    for np_ in WARP_CANDIDATES})
    fshapes.update({f"q{np_}": dict(fwd_px_per_thread=np_, fwd_blocks=L.GS_BLOCKS_QUEUE) for np_ in CANDIDATES})
    fshapes["r2"] = dict(fwd_px_per_thread=2, fwd_blocks=L.GS_BLOCKS_RING)
    fshapes["r2@64"] = dict(fwd_px_per_thread=2, fwd_blocks=L.GS_BLOCKS_RING, fwd_batch=64)
    for key, shape in fshapes.items():
        r.prm_c = dataclasses.replace(base, **shape).c()
        try:
            timings["fwd"][key] = _time(lambda: r.render_fwd(field), reps, stream)
        except L.GsError as e:
            if e.status != L.GS_ERR_UNSUPPORTED:
                raise
    best_f = min(timings["fwd"], key=timings["fwd"].get)
    fwd = dict(fshapes[best_f])
    if fwd["fwd_blocks"] != L.GS_BWD_BLOCKS_GROUP:
        # the splats staged per round by the per-tile forward, for the chosen shape ("2@64": shape 2, 64)
        best_batch = fwd.get("fwd_batch", 128)
        timings["fwd_batch"] = {best_batch: timings["fwd"][best_f]}
        for batch in BATCH_CANDIDATES:
            if batch != best_batch:
                r.prm_c = dataclasses.replace(base, **dict(fwd, fwd_batch=batch)).c()
                try:
                    timings["fwd_batch"][batch] = _time(lambda: r.render_fwd(field), reps, stream)
                except L.GsError as e:  # not built for this shape
                    if e.status != L.GS_ERR_UNSUPPORTED:
                        raise
        fwd["fwd_batch"] = min(timings["fwd_batch"], key=timings["fwd_batch"].get)
    r.prm_c = dataclasses.replace(base, **fwd).c()
    r.render_fwd(field)
    shapes = {np_: dict(bwd_px_per_thread=np_, bwd_blocks=L.GS_BWD_BLOCKS_TILE) for np_ in CANDIDATES}
    shapes.update({f"w{np_}": dict(bwd_px_per_thread=np_, bwd_blocks=L.GS_BWD_BLOCKS_GROUP)
                   for np_ in WARP_CANDIDATES})
    for key, shape in shapes.items():
        if factored and shape["bwd_blocks"] == L.GS_BWD_BLOCKS_TILE:
            continue
        r.prm_c = dataclasses.replace(base, **fwd, **shape).c()
        try:
            timings["bwd"][key] = _time(lambda: r.render_bwd(field, grad_mode, factored=factored), reps, stream)
        except L.GsError as e:
            if e.status != L.GS_ERR_UNSUPPORTED:
                raise
    best_b = min(timings["bwd"], key=timings["bwd"].get)
    tuned = dataclasses.replace(base, **fwd, **shapes[best_b])
    r.params = tuned
    r.prm_c = tuned.c()
    if verbose:
        print("autotune:", timings, "->", best_f, best_b)
    return tuned, timings
