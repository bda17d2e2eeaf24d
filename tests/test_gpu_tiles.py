"""Work-unit shapes of the batched tensor-core kernel (apc_batch_set_tiles)
and the project's tile tuner (apc_batch_autotune), through the C ABI.

Every row of a sweep-A unit and every column of a sweep-B unit is computed by
the same instructions in the same order whatever the unit's size, so all
shapes give bit-identical iterates (forward and reverse sweep); they are also
checked against the oracle's affine iteration on the BF16 bases."""
import numpy as np
import pytest

from oracle import apc_oracle as O
from paper_1708_01413_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = [(256, 512, 2, 0), (128, 512, 2, 1), (256, 128, 0, 2), (128, 256, 4, 0), (128, 128, 1, 2)]
SPLITS = [(2, 1), (1, 4), (4, 2), (8, 8)]


def _env():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1708_01413_gb300 import apc, build
    build.build()
    return apc, torch.device("cuda:0")


def _systems(k, seed):
    # sizes that leave ragged last units for every shape: n not a multiple of
    # 128 or 256, packed widths not multiples of 512
    rng = np.random.default_rng(seed)
    out = []
    for n_s in (200, 330, 700, 1100):
        A_s = rng.standard_normal((n_s, n_s)) + 0.5 * np.sqrt(n_s) * np.eye(n_s)
        out.append((A_s, rng.standard_normal((n_s, k)), inputs.uneven_offsets(n_s, 16, 128, rng)))
    return out


def _oracle_forward(systems, params, T):
    out = []
    for (A, B, o), (g, e) in zip(systems, params):
        bl = O.partition(A, B, o)
        QR = [O.block_qr(Ai) for Ai, _ in bl]
        cs = [O.block_coefficients(Q, R, bi) for (Q, R), (_, bi) in zip(QR, bl)]
        out.append(O.apc_run_affine([O.round_bf16(Q) for Q, _ in QR], cs, g, e, T)[1])
    return out


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


@pytest.mark.parametrize("k", [5, 32])
def test_every_tile_shape_gives_identical_iterates(k):
    # unit shapes, prefetch distances and L2 policies: bit-identical results;
    # units split over several CTAs (machines of sweep A, rows of sweep B):
    # the same up to the order of two FP32 sums, and the oracle within 1e-4
    apc, dev = _env()
    systems = _systems(k, 21)
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems], [o for _, _, o in systems],
                             tiles="default")
    params = [(1.0, 1.0), (1.1, 2.0), (0.9, 1.5), (1.2, 3.0)]
    bt.set_params([p[0] for p in params], [p[1] for p in params])
    G = [torch.tensor(np.random.default_rng(4).standard_normal((A.shape[0], k)), device=dev) for A, _, _ in systems]
    results = []
    for shape in SHAPES:
        bt.set_tiles(*shape)
        assert bt.tiles() == tuple(shape) + (1, 1)
        results.append((bt.forward(12), bt.x(3, 2), bt.backward(G, 7)))
    X0, xs0, DB0 = results[0]
    for shape, (X, xs, DB) in zip(SHAPES[1:], results[1:]):
        assert all(torch.equal(a, b) for a, b in zip(X, X0)), shape
        assert torch.equal(xs, xs0), shape
        assert all(torch.equal(a, b) for a, b in zip(DB, DB0)), shape
    ref = _oracle_forward(systems, params, 12)
    for x, r in zip(X0, ref):
        assert np.linalg.norm(x.cpu().numpy() - r) <= 1e-4 * np.linalg.norm(r)
    for sa, sb in SPLITS:
        for shape in (SHAPES[0], SHAPES[4]):
            bt.set_tiles(*shape, split_a=sa, split_b=sb)
            X, xs, DB = bt.forward(12), bt.x(3, 2), bt.backward(G, 7)
            assert max(_rel(a, b) for a, b in zip(X, X0)) <= 1e-5, (shape, sa, sb)
            assert _rel(xs, xs0) <= 1e-5, (shape, sa, sb)
            assert max(_rel(a, b) for a, b in zip(DB, DB0)) <= 1e-5, (shape, sa, sb)
            for x, r in zip(X, ref):
                assert np.linalg.norm(x.cpu().numpy() - r) <= 1e-4 * np.linalg.norm(r)


def test_split_units_with_heavy_ball():
    # the heavy-ball form accumulates over every machine in one buffer; split
    # into parts its gradient is summed by the last part
    apc, dev = _env()
    systems = _systems(6, 23)
    bt = apc.apc_batch_setup([torch.tensor(A, device=dev) for A, _, _ in systems],
                             [torch.tensor(B, device=dev) for _, B, _ in systems], [o for _, _, o in systems],
                             tiles="default")
    bt.set_hb_params([0.3] * 4, [0.5] * 4)
    bt.reset()
    bt.iterate(9)
    want = [bt.xbar(s) for s in range(4)]
    bt.set_tiles(128, 128, 2, 0, 4, 4)
    bt.reset()
    bt.iterate(9)
    assert max(_rel(bt.xbar(s), want[s]) for s in range(4)) <= 1e-5


def test_autotune_picks_a_candidate_and_caches_it(tmp_path):
    apc, dev = _env()
    systems = _systems(8, 22)
    As = [torch.tensor(A, device=dev) for A, _, _ in systems]
    Bs = [torch.tensor(B, device=dev) for _, B, _ in systems]
    offs = [o for _, _, o in systems]
    bt = apc.apc_batch_setup(As, Bs, offs, tiles="default")
    bt.set_params([1.0] * 4, [1.5] * 4)
    bt.reset()
    cache = str(tmp_path / "tiles.json")
    tiles, best, dflt = bt.autotune(iters=3, reps=2, cache=cache)
    assert tiles[0] in (128, 256) and tiles[1] in (128, 256, 512) and tiles[2] in (0, 1, 2, 4) and tiles[3] in (0, 1, 2)
    assert tiles[4] in (1, 2, 4, 8) and tiles[5] in (1, 2, 4, 8)
    assert 0 < best <= dflt
    assert bt.tiles() == tiles
    with pytest.raises(apc.ApcError):  # the tuning advanced the state: reset first
        bt.iterate(1)
    X = bt.forward(5)
    # a new batch with the same key reads the tuner's choice from the cache
    bt2 = apc.apc_batch_setup(As, Bs, offs, cache=cache)
    assert bt2.tiles() == tiles
    bt2.set_params([1.0] * 4, [1.5] * 4)
    X2 = bt2.forward(5)
    assert all(torch.equal(a, b) for a, b in zip(X, X2))
    assert all(np.isfinite(x.cpu().numpy()).all() for x in X)
