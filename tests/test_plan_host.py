"""Host-side segment planner of the blocked kernel (fdtd_plan_segments), run
on the CPU through the C ABI: the layout rules every plan must keep, the
segment count, and optimality of the largest estimated segment cost against
an exhaustive dynamic programme over every valid cut set. The planner has no
counterpart in the paper (it balances this implementation's warp tasks)."""
import numpy as np
import pytest

from fdtd_inputs import config_c1, config_c2, config_c3, config_c5, config_e2

# general-path cost in lean iterations, per polarisation (S, P): the weights
# the planner was tuned with on GB300
WEIGHT = {0: 12.0, 1: 8.5}
TOL = 0.25          # the planner's binary search stops within this of the optimum


@pytest.fixture(scope="module")
def fd():
    from paper_2512_17132_gb300 import build, fdtd
    build.build()
    return fdtd


def _dummy():
    return np.zeros((1, 1), np.uint8)


def _grid(fd, ny, P, js, jr, jt, nx=256):
    spec = config_c1().with_(ny=ny, pml_cells=P, tfsf_row=js, r_row=jr, t_row=jt, nx=nx,
                             labels=np.zeros((ny, nx), np.uint8))
    return fd.make_grid(spec)


def _costs(g, K, w):
    """Prefix sums C of the iteration costs, written from the planner's
    contract: iteration t costs 1 when all rows t-K..t-1 it updates lie in
    max(1, P)..ny-P-1 and none is a source or monitor row, else w."""
    ny, P = g.ny, g.pml_cells
    special = {g.tfsf_row, g.r_row, g.r_row + 1, g.t_row, g.t_row + 1}
    c = np.empty(ny + K)
    for t in range(ny + K):
        rows = range(t - K, t)
        lean = all(max(1, P) <= r <= ny - P - 1 and r not in special for r in rows)
        c[t] = 1.0 if lean else w
    return np.concatenate([[0.0], np.cumsum(c)])


def _seg_cost(C, K, y0, y1):
    return C[y1 + K] - C[0 if y0 == 0 else y0 - K]


def _valid_cuts(g, K):
    return [y for y in range(1, g.ny) if y >= K and y not in (g.r_row + 1, g.t_row + 1)]


def _optimum(g, K, n_max, w):
    """Smallest achievable largest segment cost with at most n_max segments
    (exhaustive dynamic programme over the valid cut positions)."""
    C = _costs(g, K, w)
    pos = [0] + _valid_cuts(g, K) + [g.ny]
    idx = {y: i for i, y in enumerate(pos)}
    m = len(pos)
    P0 = np.array(pos)
    # cost matrix over (start, end) of allowed boundaries
    start = np.where(P0 == 0, 0, P0 - K)
    cost = C[P0[None, :] + K] - C[start[:, None]]
    best = np.full(m, np.inf)
    best[0] = 0.0
    out = np.inf
    for _ in range(n_max):
        nxt = np.full(m, np.inf)
        for j in range(1, m):
            cand = np.maximum(best[:j], cost[:j, j])
            nxt[j] = cand.min()
        out = min(out, nxt[idx[g.ny]])
        best = nxt
    return out


def _n_target(ny, seg, K):
    # about ny / seg segments, halves rounded away from zero
    return max(1, int(np.floor(ny / max(seg, K + 1) + 0.5)))


def _check_rules(g, K, b):
    assert b[0] == 0 and b[-1] == g.ny
    assert np.all(np.diff(b) > 0)
    for y in b[1:-1]:
        assert y >= K and y != g.r_row + 1 and y != g.t_row + 1


@pytest.mark.parametrize("pol", [0, 1])
def test_random_small_grids_are_optimal(fd, pol):
    rng = np.random.default_rng(7 + pol)
    for _ in range(40):
        ny = int(rng.integers(40, 260))
        P = int(rng.integers(0, 12))
        jr = int(rng.integers(P, P + 8))
        js = jr + int(rng.integers(1, 10))
        jt = int(rng.integers(js + 1, ny - P - 2))
        K = int(rng.integers(1, 9))
        seg = int(rng.integers(max(K + 1, ny // 16), max(K + 2, ny // 2)))
        g = _grid(fd, ny, P, js, jr, jt)
        b = fd.fdtd_plan_segments(g, seg, K, pol)
        _check_rules(g, K, b)
        n_target = _n_target(ny, seg, K)
        assert len(b) - 1 <= n_target
        C = _costs(g, K, WEIGHT[pol])
        worst = max(_seg_cost(C, K, b[i], b[i + 1]) for i in range(len(b) - 1))
        opt = _optimum(g, K, n_target, WEIGHT[pol])
        assert worst <= opt + TOL, (ny, P, js, jr, jt, K, seg, worst, opt)


def _configs():
    return [config_c1(), config_c5(), config_e2(1.0),
            config_c2(labels=_dummy()), config_c3(labels=_dummy())]


@pytest.mark.parametrize("K", [1, 4, 7, 8])
def test_config_grids_keep_the_rules_and_the_count(fd, K):
    for spec in _configs():
        g = fd.make_grid(spec)
        # the shortest segments (K + 1 rows) only on the grids up to 6000 rows
        for seg in ((K + 1,) if g.ny <= 6000 else ()) + (45, 187, 370):
            for pol in (0, 1):
                b = fd.fdtd_plan_segments(g, seg, K, pol)
                _check_rules(g, K, b)
                n_target = _n_target(g.ny, seg, K)
                # enough valid cuts exist on these grids: the count is met
                assert len(b) - 1 == n_target, (spec.name, K, seg, pol, len(b) - 1)


def test_balanced_plan_beats_equal_heights(fd):
    # config 2, K = 8, the wave model's 187-row segments: the balanced plan's
    # costliest task is far cheaper than that of equal-height cuts
    g = fd.make_grid(config_c2(labels=_dummy()))
    K, seg = 8, 187
    for pol in (0, 1):
        C = _costs(g, K, WEIGHT[pol])
        b = fd.fdtd_plan_segments(g, seg, K, pol)
        n = len(b) - 1
        worst = max(_seg_cost(C, K, b[i], b[i + 1]) for i in range(n))
        eq = np.linspace(0, g.ny, n + 1).round().astype(int)
        worst_eq = max(_seg_cost(C, K, eq[i], eq[i + 1]) for i in range(n))
        mean = (C[g.ny + K] + 2 * K * (n - 1)) / n
        assert worst < 0.8 * worst_eq
        assert worst < 1.1 * mean


def test_argument_errors(fd):
    import ctypes as C
    g = fd.make_grid(config_c1())
    for K in (0, 9):
        with pytest.raises(fd.FDTDError) as e:
            fd.fdtd_plan_segments(g, 40, K, 0)
        assert e.value.code == fd.FDTD_EINVAL
    with pytest.raises(fd.FDTDError):
        fd.fdtd_plan_segments(g, 40, 8, 2)
    bad = fd.make_grid(config_c1())
    bad.t_row = bad.ny - bad.pml_cells - 1          # monitor inside the CPML margin
    with pytest.raises(fd.FDTDError) as e:
        fd.fdtd_plan_segments(bad, 40, 8, 0)
    assert "t_row" in str(e.value)
    lib = fd.load_library()
    out = (C.c_int32 * 2)()
    assert lib.fdtd_plan_segments(C.byref(g), 40, 8, 0, out, 2) == fd.FDTD_EINVAL
    assert lib.fdtd_plan_segments(None, 40, 8, 0, out, 2) == fd.FDTD_EINVAL
    # one segment when seg_rows covers the grid; the call needs no GPU
    assert list(fd.fdtd_plan_segments(g, 10 ** 6, 8, 0)) == [0, g.ny]
