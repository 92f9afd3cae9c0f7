"""A seeded sweep of small fields against the oracle's plain arithmetic.

Each case draws a field (grid shape, cell sizes, ln K variance, wells,
inactive cells), a particle set (random offsets, and particles started on
faces, edges and corners of their cells), a stop time and output times from
one seed, and runs both precisions through the C ABI:

- FP64: cell sequences, statuses, step counts and exit faces equal, times and
  positions within 1e-10 of the plain oracle, any divergent particle parted
  at a near-tie (G.compare_fp64_plain); the same bits as the mirror oracle;
- mixed precision: every particle within its per-particle bound
  (G.check_mixed).

Uniform-flow fields (A = 0 in every cell: the exit time is distance over
velocity, the limit the log form must reach) and fields with wells strong
enough to capture every particle that reaches them are part of the sweep,
and so are strongly anisotropic fields (cell sizes 1e-3 to 1e3 m across
the axes, porosity down to 0.01), whose exit times differ by orders of
magnitude between the axes of one cell.
"""
import numpy as np
import pytest

import oracle as O
from paper_2302_13590_gb300 import inputs as I
from paper_2302_13590_gb300 import mp
from tests import gpu_common as G
from tests import helpers as H

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch  # noqa: F401
    c = mp.Context(0)
    yield c
    c.close()


def _case(seed):
    rng = np.random.default_rng(7000 + seed)
    kind = seed % 4
    if kind == 3:
        f = H.uniform_x_field(int(rng.integers(1, 4)), int(rng.integers(2, 6)), int(rng.integers(4, 12)), seed=seed,
                              q_sign=1.0 if seed % 8 < 4 else -1.0)
    else:
        f = I.random_box_field(int(rng.integers(1, 5)), int(rng.integers(3, 12)), int(rng.integers(5, 16)),
                               seed=8000 + seed, lnk_var=float(rng.uniform(0.0, 3.0)), n_wells=int(rng.integers(0, 4)),
                               n_inactive=int(rng.integers(0, 4)), well_scale=float(rng.choice([0.3, 1.0, 30.0])))
    n = int(rng.choice([1, 31, 32, 33, 257, 1500]))
    ib = np.asarray(f.ibound).reshape(-1)
    act = np.nonzero(ib == 1)[0]
    cells = rng.choice(act, n).astype(np.int32)
    frac = rng.random((n, 3))
    # a share of the particles on faces, edges and corners of their cells
    on = rng.random((n, 3)) < 0.2
    frac[on] = rng.integers(0, 2, size=int(on.sum())).astype(np.float64)
    return f, cells, frac, rng


@pytest.mark.parametrize("seed", list(range(16)))
def test_sweep_against_plain_oracle(ctx, seed):
    f, cells, frac, rng = _case(seed)
    fh = ctx.field(f)
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0)
    tt = full["t"][np.isfinite(full["t"]) & (full["t"] > 0)]
    scale = float(np.median(tt)) if tt.size else 1.0
    t_stop = np.inf if seed % 3 else float(rng.uniform(0.2, 1.5)) * scale
    times = np.sort(rng.uniform(0.0, 1.2, 6)) * scale
    for sch in (mp.SCHED_STATIC, mp.SCHED_DYNAMIC):
        ep, ts, st = G.gpu_run(ctx, fh, cells=cells, frac=frac, times=times, t_stop=t_stop, schedule=sch)
        assert st["device_error"] == 0
        mirror = O.track(f, st0, t_stop=t_stop, times=times, arith="mirror")
        G.compare_fp64(ep, mirror, dmin=G.dmin(f))
        G.compare_timeseries_fp64(ts, mirror, dmin=G.dmin(f))
        plain = O.track(f, st0, t_stop=t_stop, times=times)
        G.compare_fp64_plain(ep, plain, field=f, state=st0, ts=ts, times=times, t_stop=t_stop,
                             label=f"sweep {seed}")
    epm, _, stm = G.gpu_run(ctx, fh, cells=cells, frac=frac, t_stop=t_stop, precision=mp.PREC_MIXED)
    assert stm["device_error"] == 0
    G.check_mixed(epm, field=f, state=st0, t_stop=t_stop, label=f"sweep {seed}")
    mp.mp_field_free(fh)


def _aniso_case(seed):
    rng = np.random.default_rng(9000 + seed)
    sizes = [(0.001, 0.01), (0.02, 0.1), (1.0, 5.0), (100.0, 1000.0)]
    order = rng.permutation(4)[:3]
    f = I.random_box_field(int(rng.integers(1, 4)), int(rng.integers(3, 9)), int(rng.integers(5, 12)),
                           seed=9500 + seed, lnk_var=float(rng.uniform(1.0, 4.0)), dx=sizes[order[0]],
                           dy=sizes[order[1]], dz=sizes[order[2]], porosity=(0.01, 0.3),
                           n_wells=int(rng.integers(0, 3)), n_inactive=int(rng.integers(0, 3)))
    n = int(rng.choice([33, 257, 1000]))
    act = np.nonzero(np.asarray(f.ibound).reshape(-1) == 1)[0]
    cells = rng.choice(act, n).astype(np.int32)
    frac = rng.random((n, 3))
    on = rng.random((n, 3)) < 0.2
    frac[on] = rng.integers(0, 2, size=int(on.sum())).astype(np.float64)
    return f, cells, frac, rng


@pytest.mark.parametrize("seed", list(range(6)))
def test_sweep_anisotropic(ctx, seed):
    f, cells, frac, rng = _aniso_case(seed)
    fh = ctx.field(f)
    st0 = O.release_explicit(f, cells, frac)
    full = O.track(f, st0)
    tt = full["t"][np.isfinite(full["t"]) & (full["t"] > 0)]
    scale = float(np.median(tt)) if tt.size else 1.0
    times = np.sort(rng.uniform(0.0, 1.2, 5)) * scale
    for sch in (mp.SCHED_STATIC, mp.SCHED_DYNAMIC):
        ep, ts, st = G.gpu_run(ctx, fh, cells=cells, frac=frac, times=times, schedule=sch)
        assert st["device_error"] == 0
        mirror = O.track(f, st0, times=times, arith="mirror")
        G.compare_fp64(ep, mirror, dmin=G.dmin(f))
        G.compare_timeseries_fp64(ts, mirror, dmin=G.dmin(f))
        plain = O.track(f, st0, times=times)
        G.compare_fp64_plain(ep, plain, field=f, state=st0, ts=ts, times=times, t_stop=np.inf,
                             label=f"anisotropic {seed}")
    epm, _, stm = G.gpu_run(ctx, fh, cells=cells, frac=frac, precision=mp.PREC_MIXED)
    assert stm["device_error"] == 0
    G.check_mixed(epm, field=f, state=st0, t_stop=np.inf, label=f"anisotropic {seed}")
    mp.mp_field_free(fh)
