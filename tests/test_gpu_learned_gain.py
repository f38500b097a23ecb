"""The learned Newton update end to end on the GPU: targets from the
solver's own FP64 solves, training with the BF16 tensor-core kernels, and
held-out solves from the network's prediction.  The learned start must
lower the iteration count on average, and every solve must still meet the
tolerance and match the zero-guess solution (the fallback keeps any bad
guess out)."""
import numpy as np
import pytest

import bogen
import oracle
from bogen import learned as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def bo():
    import paper_1606_00556_gb300 as m
    m.build()
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return m


def test_learned_start_reduces_iterations(bo):
    from paper_1606_00556_gb300 import learned
    ctx = bo.Context(0)
    dims = (32, 32, 16)
    V = int(np.prod(dims))
    n_train, n_test = 96, 12
    X = torch.empty(n_train, V, 16, dtype=torch.bfloat16, device="cuda")
    Y = torch.empty(n_train, V, 4, dtype=torch.float32, device="cuda")
    A = P = None
    for i, (f, a) in enumerate(L.samples(range(1000, 1000 + n_train), dims, processes=4)):
        if A is None:
            A = bo.Matrix.from_bsr(ctx, bo.grid(*dims), a["rowptr"], a["col"], a["val"])
            P = bo.Preconditioner(A)
        else:
            A.update_values(a["val"])
            P.update()
        b = torch.tensor(a["b"], device="cuda")
        x = torch.zeros_like(b)
        assert P.solve(b, x, tol=1e-10)["status"] == bo.BO_OK
        X[i] = torch.from_numpy(f).to(torch.bfloat16).cuda()
        Y[i] = torch.from_numpy(L.targets(x.cpu().numpy())).cuda()
    net = bo.CNN(ctx, *dims, max_batch=8, seed=0)
    losses = learned.train(net, X, Y, steps=400, batch=8, lr=2e-3, nout=3, log_every=50)
    assert losses[-1][1] < 0.5 * losses[0][1], losses
    it0, it1, it2, r1 = [], [], [], []
    for f, a in L.samples(range(5000, 5000 + n_test), dims, processes=4):
        Ao = oracle.BsrMatrix(a["rowptr"], a["col"], a["val"])
        A.update_values(a["val"])
        P.update()
        b = torch.tensor(a["b"], device="cuda")
        xz = torch.zeros_like(b)
        it0.append(P.solve(b, xz, tol=1e-8)["iters"])
        xf = torch.from_numpy(f).to(torch.bfloat16).cuda()[None]
        for coarse, its in ((None, it1), ((8, 8, 4), it2)):
            x = torch.empty_like(b)
            info = learned.learned_solve(P, net, xf, b, x, L.TARGET_SCALE, 3, coarse_tile=coarse)
            assert info["status"] == bo.BO_OK
            xg = x.cpu().numpy()
            assert oracle.rel_residual(Ao, a["b"], xg) <= 1e-8
            assert np.linalg.norm(xg - xz.cpu().numpy()) <= 1e-6 * np.linalg.norm(xz.cpu().numpy())
            its.append(info["iters"])
            if coarse is None:
                r1.append(info["guess_used"])
    print(f"iterations zero {np.mean(it0):.2f} learned {np.mean(it1):.2f} learned+coarse {np.mean(it2):.2f} "
          f"guess kept {np.mean(r1):.2f}")
    assert np.mean(it1) < np.mean(it0)
