"""BLR matrix times several right-hand sides (the paper's application,
Sec. 7): Y += A X through the library (diagonal T-form batch, low-rank
chains, one product per block row) against the oracle applied to the dense
matrix assembled from the blocks.  Fused and unfused chains; block rows in
one group, in uneven groups, and more groups asked for than block rows."""
import numpy as np
import pytest
import torch

import oracle
from paper_2311_07602_gb300 import blr
from paper_2311_07602_gb300 import lrbatch as L

pytestmark = pytest.mark.gpu


def dense(M):
    nb, b, r = M.nb, M.b, M.r
    D = M.D.numpy().reshape(nb, b, b).transpose(0, 2, 1)            # column-major blocks
    U = M.U.numpy().reshape(nb, (nb - 1) * r, b).transpose(0, 2, 1)  # b x (nb-1) r panels
    S = M.S.numpy().reshape(nb, nb - 1, r, r).transpose(0, 1, 3, 2)
    V = M.V.numpy().reshape(nb, nb - 1, b, r).transpose(0, 1, 3, 2)
    A = np.zeros((nb * b, nb * b))
    mag = np.zeros_like(A)
    for i in range(nb):
        A[i * b:(i + 1) * b, i * b:(i + 1) * b] = D[i]
        mag[i * b:(i + 1) * b, i * b:(i + 1) * b] = np.abs(D[i])
        for jp in range(nb - 1):
            j = jp + (jp >= i)
            Uij = U[i][:, jp * r:(jp + 1) * r]
            A[i * b:(i + 1) * b, j * b:(j + 1) * b] = Uij @ S[i, jp] @ V[i, jp]
            mag[i * b:(i + 1) * b, j * b:(j + 1) * b] = np.abs(Uij) @ np.abs(S[i, jp]) @ np.abs(V[i, jp])
    return A, mag


@pytest.mark.parametrize("fused,groups", [(True, 1), (True, 4), (False, 4), (True, 9)])
def test_blr_matvec_against_dense_oracle(fused, groups):
    nb, b, r, nrhs = 6, 48, 4, 8
    M = blr.random_blr(nb, b, r, seed=3)
    N = nb * b
    rng = np.random.default_rng(4)
    X = rng.standard_normal((N, nrhs))
    Y0 = rng.standard_normal((N, nrhs))
    A, mag = dense(M)
    Yexp = np.ascontiguousarray(Y0.ravel(order="F")).copy()
    oracle.gemm(N, nrhs, N, np.ascontiguousarray(A.ravel(order="F")), 0, N,
                np.ascontiguousarray(X.ravel(order="F")), 0, N, Yexp, 0, N)
    Yexp = Yexp.reshape(nrhs, N).T
    Md = blr.BLRMatrix(nb, b, r, *(t.to("cuda") for t in (M.D, M.U, M.S, M.V)))
    Xd = torch.tensor(X.ravel(order="F"), device="cuda")
    Yd = torch.tensor(Y0.ravel(order="F"), device="cuda")
    with L.Handle(0) as h:
        mv = blr.BLRMatVec(h, Md, Xd, Yd, nrhs, fused=fused, groups=groups)
        mv.run()
        torch.cuda.synchronize()
        mv.close()
    got = Yd.cpu().numpy().reshape(nrhs, N).T
    assert np.linalg.norm(got - Yexp) <= 1e-13 * np.linalg.norm(Yexp)
    bound = 4 * oracle.gamma(N + 3 * r + nrhs + 4) * (np.abs(Y0) + mag @ np.abs(X))
    assert np.all(np.abs(got - Yexp) <= bound)


def test_blr_full_size_sampled_rows():
    """The benchmark's product in its launch configuration (N = 65,536: 128 x
    128 blocks of 512, rank 8, 8 right-hand sides, two block-row groups);
    block rows 0, 63, 64 and 127 (both ends of both groups) recomputed by the
    oracle block by block in the same association, D_i X_i, then
    U_i [S_ij (V_ij X_j)]_j."""
    nb, b, r, nrhs = 128, 512, 8, 8
    N, K = nb * b, (nb - 1) * r
    M = blr.random_blr(nb, b, r, seed=8, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(9)
    X = torch.empty(N * nrhs, dtype=torch.float64, device="cuda").normal_(generator=g)
    Y0 = torch.empty(N * nrhs, dtype=torch.float64, device="cuda").normal_(generator=g)
    Y = Y0.clone()
    with L.Handle(0) as h:
        mv = blr.BLRMatVec(h, M, X, Y, nrhs)
        mv.run()
        torch.cuda.synchronize()
        mv.close()
    Xh, Y0h, Yh = X.cpu().numpy(), Y0.cpu().numpy(), Y.cpu().numpy()
    Xm = Xh.reshape(nrhs, N).T
    for i in (0, 63, 64, 127):
        D = M.D[i * b * b:(i + 1) * b * b].cpu().numpy()
        Up = M.U[i * b * K:(i + 1) * b * K].cpu().numpy()
        q0 = i * (nb - 1)
        S = M.S[q0 * r * r:(q0 + nb - 1) * r * r].cpu().numpy()
        V = M.V[q0 * r * b:(q0 + nb - 1) * r * b].cpu().numpy()
        exp = Y0h.reshape(nrhs, N)[:, i * b:(i + 1) * b].ravel().copy()     # b x nrhs, ld b
        oracle.gemm(b, nrhs, b, D, 0, b, Xh, i * b, N, exp, 0, b)
        T = np.zeros(K * nrhs)
        mag_t = np.zeros((K, nrhs))
        for jp in range(nb - 1):
            j = jp + (jp >= i)
            vx = np.zeros(r * nrhs)
            oracle.gemm(r, nrhs, b, V, jp * r * b, r, Xh, j * b, N, vx, 0, r)
            oracle.gemm(r, nrhs, r, S, jp * r * r, r, vx, 0, r, T, jp * r, K)
            Vb = V[jp * r * b:(jp + 1) * r * b].reshape(b, r).T
            Sb = S[jp * r * r:(jp + 1) * r * r].reshape(r, r).T
            mag_t[jp * r:(jp + 1) * r] = np.abs(Sb) @ (np.abs(Vb) @ np.abs(Xm[j * b:(j + 1) * b]))
        oracle.gemm(b, nrhs, K, Up, 0, b, T, 0, K, exp, 0, b)
        got = Yh.reshape(nrhs, N)[:, i * b:(i + 1) * b].ravel()
        assert np.linalg.norm(got - exp) <= 1e-13 * np.linalg.norm(exp), i
        mag = (np.abs(Y0h.reshape(nrhs, N)[:, i * b:(i + 1) * b].T) + np.abs(D.reshape(b, b).T) @
               np.abs(Xm[i * b:(i + 1) * b]) + np.abs(Up.reshape(K, b).T) @ mag_t)
        bound = 4 * oracle.gamma(b + K + b + r + 4) * mag
        assert np.all(np.abs(got - exp).reshape(nrhs, b).T <= bound), i
