"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module holds no part of the method's arithmetic: it only draws the
random numbers that the method consumes as inputs (Rambo uniforms, sampled
helicity labels, sampled colours, sampled colour-vector and polarisation
angles).  Both the CUDA path and the CPU oracle are
fed the arrays it returns, so that they see identical inputs.

Generator: SplitMix64 (Steele, Lea, Flood 2014) used as a counter-based
generator, value(seed, stream, i) = mix(mix(seed * GOLDEN + stream) + i *
GOLDEN), with the 53 high bits mapped to the open interval (0, 1).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

STREAM_UNIFORMS = 1
STREAM_HELICITY = 2
STREAM_COLOUR = 3
STREAM_MULTIPLICITY = 4


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def raw64(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """`count` 64-bit words of one (seed, stream) sequence starting at `offset`."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(stream))[0]
        idx = np.arange(offset, offset + count, dtype=np.uint64)
        return _mix(key + idx * _GOLDEN)


def raw64_at(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """The words of one (seed, stream) sequence at the counters `idx`."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed], dtype=np.uint64) * _GOLDEN + np.uint64(stream))[0]
        return _mix(key + np.asarray(idx, dtype=np.uint64) * _GOLDEN)


def _unit(r: np.ndarray) -> np.ndarray:
    return ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def uniforms(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in the open interval (0, 1)."""
    r = raw64(seed, stream, count, offset) >> np.uint64(11)
    return (r.astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def rambo_uniforms(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, 4(n-2)] uniforms for Rambo: per final-state gluon (u1..u4)."""
    d = 4 * (n - 2)
    return uniforms(seed, STREAM_UNIFORMS + 16 * n, batch * d, first_event * d).reshape(batch, d)


def helicities(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, n] int8 labels, +1 or -1 with equal probability."""
    r = raw64(seed, STREAM_HELICITY + 16 * n, batch * n, first_event * n) >> np.uint64(63)
    return (1 - 2 * r.astype(np.int64)).astype(np.int8).reshape(batch, n)


def adjoint_colours(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, n] int8 adjoint indices, uniform in 1..8."""
    r = raw64(seed, STREAM_COLOUR + 16 * n, batch * n, first_event * n) >> np.uint64(61)
    return (1 + r.astype(np.int64)).astype(np.int8).reshape(batch, n)


def flow_colours(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, 2n] int8 colour-flow pairs (r_i, c_i), each uniform in 1..3."""
    u = uniforms(seed, STREAM_COLOUR + 16 * n + 8, batch * 2 * n, first_event * 2 * n)
    return (1 + np.minimum((u * 3.0).astype(np.int64), 2)).astype(np.int8).reshape(batch, 2 * n)


def balanced_flow_colours(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, 2n] int8 colour-flow pairs whose column indices are a random
    permutation of the row indices (every colour appears equally often as a
    row and as a column index): uniform rows, uniformly permuted columns."""
    rows = flow_colours(n, batch, seed=seed, first_event=first_event)[:, 0::2].astype(np.int64)
    keys = raw64(seed, STREAM_COLOUR + 16 * n + 12, batch * n, first_event * n).reshape(batch, n)
    perm = np.argsort(keys, axis=1, kind="stable")
    cols = np.take_along_axis(rows, perm, axis=1)
    out = np.empty((batch, 2 * n), dtype=np.int8)
    out[:, 0::2] = rows
    out[:, 1::2] = cols
    return out


def continuous_angles(n: int, batch: int, seed: int = 0, first_event: int = 0) -> np.ndarray:
    """[batch, n, 5] float64 per gluon: cos(theta), phi, cos(theta_bar),
    phi_bar of two colour unit vectors drawn uniformly on the sphere
    (cos theta uniform in (-1, 1), phi uniform in (0, 2 pi)), and a
    polarisation angle phi_h uniform in (0, 2 pi)."""
    u = uniforms(seed, STREAM_COLOUR + 16 * n + 4, batch * n * 5, first_event * n * 5).reshape(batch, n, 5)
    out = np.empty_like(u)
    out[:, :, 0] = 2.0 * u[:, :, 0] - 1.0
    out[:, :, 2] = 2.0 * u[:, :, 2] - 1.0
    out[:, :, 1] = 2.0 * np.pi * u[:, :, 1]
    out[:, :, 3] = 2.0 * np.pi * u[:, :, 3]
    out[:, :, 4] = 2.0 * np.pi * u[:, :, 4]
    return out


def multiplicities(batch: int, n_min: int, n_max: int, seed: int = 0) -> np.ndarray:
    """[batch] int32 multiplicities uniform in n_min..n_max."""
    u = uniforms(seed, STREAM_MULTIPLICITY, batch)
    span = n_max - n_min + 1
    return (n_min + np.minimum((u * span).astype(np.int64), span - 1)).astype(np.int32)


def mixed_events(batch: int, n_min: int, n_max: int, seed: int = 0, colours: str = "adjoint") -> dict:
    """A mixed-multiplicity batch in the padded layout of the mixed plan.

    Event e has multiplicity nev[e] (multiplicities()); its uniforms,
    helicities and colours are the row e of rambo_uniforms(n, ...),
    helicities(n, ...) and adjoint_colours / flow_colours /
    balanced_flow_colours(n, ...) for that n (the generator is counter-based,
    so event e draws the same numbers as in a single-multiplicity batch that
    contains it at position e).  Returns nev [B] int32, u [B, 4(n_max-2)]
    float64 (columns past 4(n_e-2) are 0.5), hel [B, n_max] int8 (columns
    past n_e are +1), colors [B, 2 n_max] int8 (columns past the event's
    colour labels are 1)."""
    nev = multiplicities(batch, n_min, n_max, seed=seed)
    dmax = 4 * (n_max - 2)
    u = np.full((batch, dmax), 0.5)
    hel = np.ones((batch, n_max), dtype=np.int8)
    col = np.ones((batch, 2 * n_max), dtype=np.int8)
    for n in range(n_min, n_max + 1):
        idx = np.nonzero(nev == n)[0].astype(np.uint64)
        if idx.size == 0:
            continue
        d = 4 * (n - 2)
        cnt = (idx[:, None] * np.uint64(d) + np.arange(d, dtype=np.uint64)[None, :])
        u[idx.astype(np.int64), :d] = _unit(raw64_at(seed, STREAM_UNIFORMS + 16 * n, cnt))
        cnt = idx[:, None] * np.uint64(n) + np.arange(n, dtype=np.uint64)[None, :]
        r = raw64_at(seed, STREAM_HELICITY + 16 * n, cnt) >> np.uint64(63)
        hel[idx.astype(np.int64), :n] = (1 - 2 * r.astype(np.int64)).astype(np.int8)
        if colours == "adjoint":
            r = raw64_at(seed, STREAM_COLOUR + 16 * n, cnt) >> np.uint64(61)
            col[idx.astype(np.int64), :n] = (1 + r.astype(np.int64)).astype(np.int8)
        elif colours in ("flow", "balanced_flow"):
            c2 = idx[:, None] * np.uint64(2 * n) + np.arange(2 * n, dtype=np.uint64)[None, :]
            uu = _unit(raw64_at(seed, STREAM_COLOUR + 16 * n + 8, c2))
            fl = (1 + np.minimum((uu * 3.0).astype(np.int64), 2)).astype(np.int8)
            if colours == "balanced_flow":
                rows = fl[:, 0::2].astype(np.int64)
                keys = raw64_at(seed, STREAM_COLOUR + 16 * n + 12, cnt)
                perm = np.argsort(keys, axis=1, kind="stable")
                fl[:, 1::2] = np.take_along_axis(rows, perm, axis=1).astype(np.int8)
            col[idx.astype(np.int64), :2 * n] = fl
        else:
            raise ValueError(f"unknown colour sampling {colours!r}")
    return {"nev": nev, "u": u, "hel": hel, "colors": col}
