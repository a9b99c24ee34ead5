"""The timed path of bench.py, at its full size, checked against the oracle.

The bench's step on the two-wavelength 256x256 workload: CNN prediction (the
network with its PCA offset per wavelength, orthonormalised on the device)
into the subspace [PCA-20 of the wavelength | CNN-8], then one batched
complex64 augmented GMRES(200) solve of both wavelengths, FP64 refinement, the
step loop as a CUDA graph, a restart policy per wavelength (1300 nm: the
PCA-20 columns kept after the first cycle; 1550 nm: plain GMRES after it);
both storages of the Krylov basis.  For every solve the
true relative residual is recomputed with the oracle's sparse operator
(<= 1e-6) and the field compared with the oracle's direct solution (relative
L2 <= 1e-5).  The network is trained only briefly: the accuracy of the result
does not depend on the quality of the subspace, only the step count does.
"""
import argparse

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fdfd

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import bench  # noqa: E402
import paper_1902_00090_gb300 as ddg  # noqa: E402


@pytest.fixture(scope="module")
def setup():
    grids = bench.splitter_grids()
    g0 = grids[0]
    src = (g0.i_src, g0.sigma_src, g0.j_src)
    train_eps = np.concatenate([bench.trajectory(t)[:8] for t in range(3)])
    train_ops = {g.wavelength: [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in train_eps]
                 for g in grids}
    b_of = {g.wavelength: ddg.fdfd_source(train_ops[g.wavelength][0], *src) for g in grids}
    ctx = ddg.Context()
    U_base, U_pca = {}, {}
    for g in grids:
        lam = g.wavelength
        xs, inf, st = ddg.gmres_solve_batched(ctx, train_ops[lam], [b_of[lam]] * len(train_eps), tol=1e-6,
                                              restart=200, maxit=20000, precision="c64")
        assert st == 0
        U_base[lam], _ = ddg.pca_fit(ctx, torch.stack(xs), 8)
        U_pca[lam], _ = ddg.pca_fit(ctx, torch.stack(xs), 20)
    args = argparse.Namespace(cnn_k=8, cnn_batch=4, cnn_lr=3e-4, cnn_steps=20)
    P = bench.train_cnn(ddg, args, grids, train_ops, b_of, U_base, src, g0.D)
    test_eps = bench.trajectory(bench.N_TRAIN_TRAJ)[:4]
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for g in grids for e in test_eps]
    bs = [ddg.fdfd_source(op, *src) for op in ops]
    probs = [(g, e) for g in grids for e in test_eps]
    direct = [spla.spsolve(fdfd.operator_for(g, e).tocsc(), fdfd.source_for(g)) for g, e in probs]
    return dict(grids=grids, src=src, P=P, ops=ops, bs=bs, probs=probs, direct=direct,
                U_pca=[U_pca[g.wavelength] for g, _ in probs])


def headline_context(basis="f32"):
    ctx = ddg.Context()
    ctx.set_graphs(True)
    ctx.set_basis_storage(basis)
    ctx.set_augmented_policy(1, keep=20, wavelength=1300e-9)
    ctx.set_augmented_policy(1, keep=0, wavelength=1550e-9)
    return ctx


def headline_subspace(S):
    Ucnn = S["P"].predict(S["ops"], S["src"])
    return Ucnn, [torch.cat([up, uc]) for up, uc in zip(S["U_pca"], Ucnn)]


@pytest.mark.parametrize("basis", ["f32", "f16"])
def test_timed_step_matches_the_oracle(setup, basis):
    S = setup
    ctx = headline_context(basis)
    Ucnn, U = headline_subspace(S)
    for u in Ucnn:                                        # K13: orthonormal on the device
        uh = u.cpu().numpy()
        assert np.max(np.abs(uh.conj() @ uh.T - np.eye(8))) <= 1e-10
    xs, infos, st = ddg.augmented_gmres_solve_batched(ctx, S["ops"], S["bs"], U, tol=1e-6, restart=200,
                                                      maxit=5000, precision="c64")
    assert st == 0, infos
    for (g, e), x, xd, inf in zip(S["probs"], xs, S["direct"], infos):
        A = fdfd.operator_for(g, e)
        b = fdfd.source_for(g)
        xh = x.cpu().numpy()
        res = np.linalg.norm(b - A @ xh) / np.linalg.norm(b)
        assert res <= 1e-6, (g.wavelength, res, inf)
        assert abs(res - inf["true_rel_residual"]) <= 1e-9      # the library's own FP64 residual
        assert np.linalg.norm(xh - xd) / np.linalg.norm(xd) <= 1e-5, (g.wavelength, inf)
        assert inf["first_step_rel_residual"] < 1.0


def test_host_buffer_entry_point_matches_the_device_path(setup):
    # fdfd_solve_host: the same step from host permittivities to host fields
    S = setup
    ctx = headline_context()
    grids = [g for g, _ in S["probs"]]
    eps_h = [torch.from_numpy(np.ascontiguousarray(e)).pin_memory() for _, e in S["probs"]]
    x_h = [torch.empty(g.D, dtype=torch.complex128).pin_memory() for g in grids]
    infos, st = ddg.fdfd_solve_host(ctx, grids, eps_h, S["src"], x_h, P=S["P"], U_fixed=S["U_pca"], tol=1e-6,
                                    restart=200, maxit=5000, precision="c64")
    assert st == 0
    _, U = headline_subspace(S)
    xs, infos_d, _ = ddg.augmented_gmres_solve_batched(ctx, S["ops"], S["bs"], U, tol=1e-6, restart=200,
                                                       maxit=5000, precision="c64")
    for xh, xd, i1, i2 in zip(x_h, xs, infos, infos_d):
        assert i1["iters"] == i2["iters"]
        assert torch.equal(xh, xd.cpu())
