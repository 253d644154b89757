"""Comparison helpers for the GPU-vs-oracle parity tests.

Tolerances: the CUDA path computes in FP32 and must match the FP64 oracle per
step from an identical state to a relative error of 1e-5 on the field
(denominator max(|C_ref|, 1e-6 max|C_ref|)) and on cone positions
(denominator max(|p_ref|, 1) in grid units).

Cone decisions that FP32 rounding can legitimately flip are excluded and
counted: a gradient norm within 1% of grad_eps, a trial position within a
small margin of a wall, or a squared distance to a source within a small
margin of stop_radius^2.
"""
import numpy as np

import oracle

FIELD_RTOL = 1e-5
POS_RTOL = 1e-5


def field_rel_err(gpu, ref):
    ref = np.asarray(ref, np.float64)
    gpu = np.asarray(gpu, np.float64)
    scale = np.abs(ref).max()
    denom = np.maximum(np.abs(ref), 1e-6 * scale if scale > 0 else 1e-30)
    return float((np.abs(gpu - ref) / denom).max()) if ref.size else 0.0


def pos_rel_err(gpu, ref):
    """Per-cone relative position error, shape (n,)."""
    gpu = np.asarray(gpu, np.float64)
    ref = np.asarray(ref, np.float64)
    denom = np.maximum(np.linalg.norm(ref, axis=0), 1.0)
    return np.abs(gpu - ref).max(axis=0) / denom


def grid_of(w):
    return oracle.Grid(w.dim, w.nx, w.ny, w.nz if w.dim == 3 else 1, h=w.h, D=w.D, lam=w.lam, dt=w.dt)


def cone_of(w):
    return oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, w.stop_radius, w.grad_eps,
                       w.wall_mode, w.seed)


def ambiguous_cones(w, C, step, pos, dir, active, margin=1e-4):
    """Boolean mask of cones whose step-`step` decision FP32 rounding may flip."""
    g = grid_of(w)
    n = active.shape[0]
    amb = np.zeros(n, bool)
    if n == 0:
        return amb
    p = np.asarray(pos, np.float64)
    grads = oracle.gradient_at(g, C, p.T)[:, : w.dim]
    gn = np.linalg.norm(grads, axis=1)
    if w.grad_eps > 0:
        amb |= np.abs(gn - w.grad_eps) <= 0.01 * w.grad_eps
    # trial move: the clamp mode returns the unclipped direction d'
    free = oracle.Cone(w.w_prev, w.w_grad, w.w_noise, w.step_len, 0.0, w.grad_eps, 1, w.seed)
    _, d_trial, _ = oracle.cone_step(g, free, C, step, p, dir, np.ones(n, np.uint8))
    trial = p + w.step_len * d_trial
    hi = np.array([(e - 1) * w.h for e in (w.nx, w.ny, w.nz)[: w.dim]])[:, None]
    scale = np.maximum(np.linalg.norm(p, axis=0), 1.0)
    wall_gap = np.minimum(np.abs(trial), np.abs(trial - hi)).min(axis=0)
    amb |= wall_gap <= margin * scale
    if w.stop_radius > 0 and w.n_src > 0:
        cells = w.src_cell.astype(np.int64)
        xs = [(cells % w.nx) * w.h, ((cells // w.nx) % w.ny) * w.h, (cells // (w.nx * w.ny)) * w.h]
        xs = np.stack(xs[: w.dim])                              # (dim, n_src)
        d2 = ((trial[:, :, None] - xs[:, None, :]) ** 2).sum(0)  # (n, n_src)
        r2 = w.stop_radius ** 2
        amb |= (np.abs(d2 - r2) <= margin * r2 * 10).any(axis=1)
    amb &= active.astype(bool)
    return amb


def compare_cones(w, C, step, pos0, dir0, act0, got_pos, got_dir, got_act):
    """One cone step of the GPU (got_*) against the oracle's from the same state (C, pos0, dir0,
    act0 at Philox step `step`): stop flags identical, positions to POS_RTOL, directions to 1e-5,
    cones whose decision rounding may flip excluded (at most 1%, or 2) and counted."""
    want_pos, want_dir, want_act = oracle.cone_step(grid_of(w), cone_of(w), C.astype(np.float64), step,
                                                    pos0, dir0, act0, w.src_cell)
    amb = ambiguous_cones(w, C.astype(np.float64), step, pos0, dir0, act0)
    keep = ~amb
    assert amb.sum() <= max(2, 0.01 * act0.sum()), amb.sum()
    np.testing.assert_array_equal(got_act[keep], want_act[keep])
    err = pos_rel_err(got_pos[:, keep], want_pos[:, keep])
    assert (err.max() if err.size else 0.0) <= POS_RTOL, err.max()
    derr = np.abs(got_dir[:, keep] - want_dir[:, keep]).max() if keep.any() else 0.0
    assert derr <= 1e-5, derr
    return int(amb.sum())
