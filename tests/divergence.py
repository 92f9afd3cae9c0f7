"""Where two evaluations of one particle path part, and by how much they had
to disagree there.

The oracle's two arithmetic modes evaluate the same solution with different
rounding (a few ulp per step).  On a particle whose cell sequences differ,
the first cell-step at which the two traces choose differently is one of:

- ``axis``: both leave the cell, through faces of different axes; the gap is
  the difference of the two competing exit times in the reference trace;
- ``face``: the same axis, opposite faces (the particle velocity changes
  sign between the two evaluations); the gap is the reference's velocity on
  that axis, against the larger face velocity of the axis;
- ``stop``: one reaches the stop time inside the cell, the other leaves it;
  the gap is the distance of the reference's step end from the stop time
  (where one leaves and the other has no reachable face on that axis, the
  kind is ``face``);
- ``cell``: the same exit, different cells entered (a quadtree hand-over);
- ``end``: the traces agree step by step but one ends earlier (a status
  decided differently after the last common step).

The gap is measured against a scale (the time at the end of the step, or the
face velocity), so ``gap <= rtol * scale`` says that the two choices cannot be
told apart at the relative tolerance the results are compared at.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

import oracle as O


@dataclass
class Divergence:
    particle: int
    step: int
    kind: str
    gap: float
    scale: float

    @property
    def rel(self) -> float:
        return self.gap / self.scale if self.scale > 0 else (0.0 if self.gap == 0 else np.inf)


def first_divergence(ref, other, t_stop=np.inf, particle=-1) -> Divergence:
    """Compare two TRACE_RECORD arrays of one particle (``ref`` the reference
    evaluation) and classify the first step at which they choose differently."""
    n = min(ref.size, other.size)
    for s in range(n):
        a, b = ref[s], other[s]
        if a["cell"] != b["cell"]:
            return Divergence(particle, s, "cell", 0.0, 1.0)
        ax_a, ax_b = int(a["ax"]), int(b["ax"])
        if ax_a == ax_b and (ax_a < 0 or a["face"][ax_a] == b["face"][ax_b]):
            continue
        t = float(a["t"])
        if ax_a >= 0 and ax_b >= 0 and ax_a != ax_b:
            ta, tb = float(a["te"][ax_a]), float(a["te"][ax_b])
            if np.isfinite(tb):
                return Divergence(particle, s, "axis", abs(tb - ta), t + tb)
            # the other evaluation's axis has no reachable face here: its
            # particle velocity changed sign
            return Divergence(particle, s, "face", abs(float(a["vp"][ax_b])), float(a["vf"][ax_b]))
        if ax_a >= 0 and ax_b >= 0:
            return Divergence(particle, s, "face", abs(float(a["vp"][ax_a])), float(a["vf"][ax_a]))
        # one leaves the cell, the other does not: either the other has no
        # reachable face on that axis (its particle velocity vanished or
        # changed sign) or it reached the stop time first
        ax = ax_a if ax_a >= 0 else ax_b
        te, te_b = float(a["te"][ax]), float(b["te"][ax])
        if not (np.isfinite(te) and np.isfinite(te_b)):
            return Divergence(particle, s, "face", abs(float(a["vp"][ax])), float(a["vf"][ax]))
        return Divergence(particle, s, "stop", abs(t + te - t_stop), float(t_stop))
    return Divergence(particle, n, "end", np.inf, 1.0)


def analyse(field, state, which, *, t_stop=np.inf, times=None, ref="plain", other="mirror", **kw):
    """Trace particles ``which`` of ``state`` in both arithmetic modes and
    return one Divergence per particle (kind ``end`` with an infinite gap
    where the traces agree step by step but end differently)."""
    out = []
    for q in np.asarray(which, dtype=np.int64):
        s1 = O.subset(state, [int(q)])
        ta = O.track(field, s1, t_stop=t_stop, times=times, arith=ref, trace=True, **kw)["trace"]
        tb = O.track(field, s1, t_stop=t_stop, times=times, arith=other, trace=True, **kw)["trace"]
        out.append(first_divergence(ta, tb, t_stop=t_stop, particle=int(q)))
    return out


def first_time_split(ref, other, rtol):
    """Two TRACE_RECORD arrays of one particle that take the same cells:
    the first step whose chosen exit time differs by more than ``rtol`` of
    the time at the end of the step, and there the particle velocity on the
    exit axis relative to its face velocity (a value near zero means the exit
    starts from a stagnation surface, where the exit time, ln(v_exit / v_p)
    / A, is set by the rounding of a vanishing v_p).  Returns (step,
    |v_p| / v_face) or (-1, inf) when no step differs."""
    for s in range(min(ref.size, other.size)):
        a, b = ref[s], other[s]
        ax = int(a["ax"])
        if ax < 0 or int(b["ax"]) != ax:
            continue
        ta, tb = float(a["te"][ax]), float(b["te"][ax])
        if abs(ta - tb) > rtol * (float(a["t"]) + max(ta, tb)):
            return s, abs(float(a["vp"][ax])) / max(float(a["vf"][ax]), 1e-300)
    return -1, float("inf")


def stagnation_exits(field, state, which, *, rtol, t_stop=np.inf, times=None, **kw):
    """For particles ``which`` (same cell sequence in both arithmetic modes,
    results further apart than ``rtol``): (particle, step, |v_p| / v_face) at
    the first step whose exit times part."""
    out = []
    for q in np.asarray(which, dtype=np.int64):
        s1 = O.subset(state, [int(q)])
        ta = O.track(field, s1, t_stop=t_stop, times=times, arith="plain", trace=True, **kw)["trace"]
        tb = O.track(field, s1, t_stop=t_stop, times=times, arith="mirror", trace=True, **kw)["trace"]
        out.append((int(q),) + first_time_split(ta, tb, rtol))
    return out
