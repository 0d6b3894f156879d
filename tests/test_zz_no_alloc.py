"""The allocation-free training step (icrs_mlp_train_step_noalloc, static
scratch inside the library) against the workspace entry point: two steps in a
row from the same state give bit-identical parameters, moments, gradients and
losses.  This file is collected last; it passes on its own and after the other
GPU tests."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_02639_gb300 import build as B
    B.build()
    from paper_2510_02639_gb300 import icrs
    return icrs


def state(G, seed):
    import torch
    from paper_2510_02639_gb300 import surrogate as SG
    th = torch.tensor(SG.init_theta(seed), device="cuda")
    return th, torch.zeros_like(th), torch.zeros_like(th), G.mlp_pack(th)


def test_noalloc_matches_workspace_step_twice(G):
    import torch
    rng = np.random.default_rng(11)
    n = 3000  # 24 tiles, ragged
    f = np.zeros((n, 8), dtype=np.float32)
    f[:, :7] = rng.uniform(-1, 1, (n, 7))
    y = rng.standard_normal(n).astype(np.float32)
    feat = torch.tensor(f, device="cuda"); tgt = torch.tensor(y, device="cuda")
    a = state(G, 3)
    b = state(G, 3)
    ga, gb = torch.zeros_like(a[0]), torch.zeros_like(b[0])
    la, lb = torch.zeros(1, device="cuda"), torch.zeros(1, device="cuda")
    ws = G.mlp_workspace(n)
    for step in (1, 2):
        G.mlp_train_step(a[0], a[1], a[2], a[3], step, 1e-3, feat, tgt, workspace=ws, grad=ga, loss=la)
        G.mlp_train_step_noalloc(b[0], b[1], b[2], b[3], step, 1e-3, feat, tgt, grad=gb, loss=lb)
        torch.cuda.synchronize()
        for x, z in zip(a, b):
            assert torch.equal(x, z)
        assert torch.equal(ga, gb) and torch.equal(la, lb)
        assert torch.isfinite(ga).all() and float(ga.abs().sum()) > 0


def test_noalloc_rejects_oversize(G):
    import torch
    th, m, v, pack = state(G, 4)
    n = G.MLP_STATIC_MAX_N + 1
    feat = torch.zeros((n, 8), dtype=torch.float32, device="cuda")
    tgt = torch.zeros((n,), dtype=torch.float32, device="cuda")
    with pytest.raises(G.IcrsError):
        G.mlp_train_step_noalloc(th, m, v, pack, 1, 1e-3, feat, tgt)
