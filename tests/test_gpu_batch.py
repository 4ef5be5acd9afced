"""Ragged batches of independent 1D Euler tubes in one persistent launch,
against the oracle run tube by tube.  FP64: every tube bit-identical to the
oracle (state, steps, final time) for every group size; FP32: within the FP32
tolerance of the oracle; both against the exact Riemann solution."""
import numpy as np
import pytest

import oracle
from oracle import riemann
from paper_1808_00037_gb300 import binding as B
from paper_1808_00037_gb300 import inputs as I

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def small_batch(seed=3, ntubes=24, nmin=30, nmax=300):
    return I.riemann_tube_batch(seed, ntubes, nmin, nmax)


def oracle_tubes(U, offsets, dx, t_end, cfl, max_steps=1 << 30):
    out = U.copy()
    steps, ts = [], []
    for t in range(len(dx)):
        a, b = offsets[t], offsets[t + 1]
        Uo, s, tt, st = oracle.run_1d(oracle.SYS_EULER1D, U[:, a:b], dx[t], t_end=t_end, cfl=cfl, bc=(1, 1),
                                      max_steps=max_steps)
        assert st == 0
        out[:, a:b] = Uo
        steps.append(s)
        ts.append(tt)
    return out, np.array(steps), np.array(ts)


def ctx(n, prec=B.T7_F64):
    return B.Context(B.T7_EULER1D, n, 1.0, prec=prec, bc=(1, 1, 0, 0))


@pytest.fixture(scope="module")
def small_ref():
    U, off, dx, _ = small_batch()
    return (U, off, dx) + oracle_tubes(U, off, dx, 0.1, 0.5)


@pytest.mark.parametrize("group", [1, 2, 4, 8])
def test_batch_f64_bitexact(small_ref, group):
    U, off, dx, Uo, so, to = small_ref
    c = ctx(U.shape[1])
    Ug = torch.tensor(U, dtype=torch.float64, device="cuda")
    steps, t = c.batch_run(Ug, off, dx, 0.1, 0.5, group_warps=group)
    assert np.array_equal(steps, so) and np.array_equal(t, to)
    assert np.array_equal(Ug.cpu().numpy(), Uo)


def test_batch_f32_against_oracle_and_exact():
    U, off, dx, states = small_batch(seed=4, ntubes=16, nmin=200, nmax=400)
    Uo, so, to = oracle_tubes(U, off, dx, 0.1, 0.5)
    c = ctx(U.shape[1], prec=B.T7_F32)
    Ug = torch.tensor(U, dtype=torch.float32, device="cuda")
    steps, t = c.batch_run(Ug, off, dx, 0.1, 0.5)
    got = Ug.double().cpu().numpy()
    assert np.allclose(t, 0.1, atol=1e-12)
    for k in range(len(dx)):
        a, b = off[k], off[k + 1]
        rng_rho = np.ptp(Uo[0, a:b]) + 1e-12
        assert np.mean(np.abs(got[0, a:b] - Uo[0, a:b])) / rng_rho < 2e-3, k
        x = (np.arange(b - a) + 0.5) / (b - a)
        rho, _, _ = riemann.sample(tuple(states[k, 0]), tuple(states[k, 1]), (x - 0.5) / 0.1)
        assert np.mean(np.abs(got[0, a:b] - rho)) / (np.ptp(rho) + 1e-12) < 5e-2, k


def test_batch_config_sample_f64():
    """The 4096-tube configuration (lengths U[256, 8192], seed 7): its shortest
    tubes run to t = 0.1 and one long tube for 20 steps, bit-identical to the
    oracle (the whole batch would take the oracle hours)."""
    U, off, dx, _ = I.riemann_tube_batch(7, 4096, 256, 8192)
    n = np.diff(off)
    pick = list(np.argsort(n, kind="stable")[:6])
    sub_off = np.concatenate([[0], np.cumsum(n[pick])])
    sub = np.concatenate([U[:, off[t]:off[t + 1]] for t in pick], axis=1)
    Uo, so, to = oracle_tubes(sub, sub_off, dx[pick], 0.1, 0.5)
    c = ctx(sub.shape[1])
    Ug = torch.tensor(sub, dtype=torch.float64, device="cuda")
    steps, t = c.batch_run(Ug, sub_off, dx[pick], 0.1, 0.5)
    assert np.array_equal(steps, so) and np.array_equal(Ug.cpu().numpy(), Uo)
    # one of the longest tubes, 20 steps
    big = int(np.argmax(n))
    Ub = np.ascontiguousarray(U[:, off[big]:off[big + 1]])
    Uo, so, to = oracle_tubes(Ub, np.array([0, Ub.shape[1]]), dx[big:big + 1], 0.1, 0.5, max_steps=20)
    c = ctx(Ub.shape[1])
    Ug = torch.tensor(Ub, dtype=torch.float64, device="cuda")
    steps, t = c.batch_run(Ug, np.array([0, Ub.shape[1]]), dx[big:big + 1], 0.1, 0.5, max_steps=20)
    assert steps[0] == 20 and np.array_equal(Ug.cpu().numpy(), Uo)


def test_batch_full_config_f32_runs_to_t_end():
    """All 4096 tubes in FP32 to t = 0.1 in one launch: every tube reaches t_end,
    mass in every tube changes only by the boundary fluxes (bounded), no error."""
    U, off, dx, _ = I.riemann_tube_batch(7, 4096, 256, 8192)
    c = ctx(U.shape[1], prec=B.T7_F32)
    Ug = torch.tensor(U, dtype=torch.float32, device="cuda")
    g, ms = c.batch_autotune(Ug, off, dx, 0.5, trial_steps=2)
    assert g in (1, 2, 4, 8) and np.all(ms > 0)
    steps, t = c.batch_run(Ug, off, dx, 0.1, 0.5)
    assert np.allclose(t, 0.1, atol=1e-12) and np.all(steps > 0)
    got = Ug.double().cpu().numpy()
    assert np.all(np.isfinite(got)) and np.all(got[0] > 0)


def test_batch_full_config_f32_close_to_f64_after_50_steps():
    """Every tube of the 4096-tube batch, 50 steps in FP32 and FP64: per tube and
    variable, the FP32 state is within 2e-4 of the FP64 state in mean absolute
    difference relative to the tube's range of that variable (pointwise, a
    stencil decision taken differently at a shock moves one cell by a few
    percent of the jump, so the pointwise bound only excludes blow-ups)."""
    U, off, dx, _ = I.riemann_tube_batch(7, 4096, 256, 8192)
    out = {}
    for prec, dtype in ((B.T7_F64, torch.float64), (B.T7_F32, torch.float32)):
        c = ctx(U.shape[1], prec=prec)
        Ug = torch.tensor(U, dtype=dtype, device="cuda")
        c.batch_run(Ug, off, dx, 0.1, 0.5, max_steps=50)
        out[prec] = Ug.double().cpu().numpy()
    d = np.abs(out[B.T7_F32] - out[B.T7_F64])
    for k in range(3):
        for t in range(0, 4096, 1):
            a, b = off[t], off[t + 1]
            rng = np.ptp(out[B.T7_F64][k, a:b]) + np.abs(out[B.T7_F64][k, a:b]).max() * 1e-3
            assert d[k, a:b].mean() <= 2e-4 * rng and d[k, a:b].max() <= 0.1 * rng, (k, t)


def test_batch_autotune_leaves_state_and_rejects_bad_offsets():
    U, off, dx, _ = small_batch()
    c = ctx(U.shape[1])
    Ug = torch.tensor(U, dtype=torch.float64, device="cuda")
    g, ms = c.batch_autotune(Ug, off, dx, 0.5, trial_steps=2)
    assert np.array_equal(Ug.cpu().numpy(), U)
    bad = off.copy()
    bad[-1] += 1
    with pytest.raises(B.T7Error) as ei:
        c.batch_run(Ug, bad, dx, 0.1, 0.5)
    assert ei.value.status == B.T7_EINVAL


def test_batch_whole_cta_phase_f64_bitexact():
    """The two-phase schedule (group_warps < 0): 1500 short tubes (30-90 cells)
    and 3 long ones (1200-1500) to t = 0.02 or 12 steps.  With G = 4 only the
    long tubes run first on whole CTAs; with G = 1 most short tubes do too, so
    both phases and the hand-over between them carry tubes.  Every tube is
    bit-identical to the oracle (state, steps, final time), so no tube is
    skipped or advanced twice."""
    Us, offs, dxs, _ = I.riemann_tube_batch(11, 1500, 30, 90)
    Ul, offl, dxl, _ = I.riemann_tube_batch(12, 3, 1200, 1500)
    cut = int(offs[700])
    U = np.concatenate([Us[:, :cut], Ul, Us[:, cut:]], axis=1)
    n = np.concatenate([np.diff(offs)[:700], np.diff(offl), np.diff(offs)[700:]])
    off = np.concatenate([[0], np.cumsum(n)])
    dx = np.concatenate([dxs[:700], dxl, dxs[700:]])
    Uo, so, to = oracle_tubes(U, off, dx, 0.02, 0.5, max_steps=12)
    assert 0 < np.sum(so < 12) < len(so)  # some tubes stop at t_end, others at max_steps
    for group in (-4, -1):
        c = ctx(U.shape[1])
        Ug = torch.tensor(U, dtype=torch.float64, device="cuda")
        steps, t = c.batch_run(Ug, off, dx, 0.02, 0.5, max_steps=12, group_warps=group)
        assert np.array_equal(steps, so) and np.array_equal(t, to), group
        assert np.array_equal(Ug.cpu().numpy(), Uo), group


@pytest.mark.parametrize("group", [3, -3, 16, -16])
def test_batch_rejects_bad_group(group):
    U, off, dx, _ = small_batch()
    c = ctx(U.shape[1])
    Ug = torch.tensor(U, dtype=torch.float64, device="cuda")
    with pytest.raises(B.T7Error) as ei:
        c.batch_run(Ug, off, dx, 0.1, 0.5, group_warps=group)
    assert ei.value.status == B.T7_EINVAL
    assert np.array_equal(Ug.cpu().numpy(), U)
