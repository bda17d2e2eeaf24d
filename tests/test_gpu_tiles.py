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


@pytest.mark.parametrize("k", [5, 32])
def test_every_tile_shape_gives_identical_iterates(k):
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
        assert bt.tiles() == shape
        X = bt.forward(12)
        xs = bt.x(3, 2)
        DB = bt.backward(G, 7)
        results.append((X, xs, DB))
    X0, xs0, DB0 = results[0]
    for shape, (X, xs, DB) in zip(SHAPES[1:], results[1:]):
        assert all(torch.equal(a, b) for a, b in zip(X, X0)), shape
        assert torch.equal(xs, xs0), shape
        assert all(torch.equal(a, b) for a, b in zip(DB, DB0)), shape
    for (A, B, o), (g, e), x in zip(systems, params, X0):
        bl = O.partition(A, B, o)
        QR = [O.block_qr(Ai) for Ai, _ in bl]
        cs = [O.block_coefficients(Q, R, bi) for (Q, R), (_, bi) in zip(QR, bl)]
        _, ref = O.apc_run_affine([O.round_bf16(Q) for Q, _ in QR], cs, g, e, 12)
        assert np.linalg.norm(x.cpu().numpy() - ref) <= 1e-4 * np.linalg.norm(ref)


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
