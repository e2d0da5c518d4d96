"""Differentiation: the flux VJP behind torch.autograd.Function.

Checked against the transposed analytic Jacobian of the FP64 oracle
(A_d(U)^T G at every point, 1e-12 * S), against central finite differences of
the GPU flux (h = 1e-6 in FP64) on 4,096 sampled points, and, at the size of
the differentiation workload (N = 2^24), against the oracle everywhere.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1809_09851_gb300 import autograd, blocks, synth

pytestmark = pytest.mark.gpu
G_ = 1.4
DEV = "cuda:0"


def _field(n, D=3, seed=1809):
    V = synth.euler3d(n, seed=seed, D=D)
    return oracle.cons_from_prim(D, G_, V)


def _dev(planes, dtype=torch.float64):
    return [torch.from_numpy(p).to(DEV).to(dtype) for p in planes]


@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
@pytest.mark.parametrize("D", [1, 2, 3])
def test_autograd_matches_transposed_jacobian(D, dw):
    n = 5003
    U = _field(n, D)
    Gc = synth.cotangent(n, D + 2)
    for d in range(D):
        Ud = [u.requires_grad_() for u in _dev(U)]
        F = autograd.flux(Ud, d, G_, dw=dw)
        loss = sum((f * g).sum() for f, g in zip(F, _dev(Gc)))
        loss.backward()
        got = [u.grad.cpu().numpy() for u in Ud]
        ref, S = oracle.flux_vjp(D, d, G_, U, Gc, scale=True)
        for k in range(D + 2):
            assert np.all(np.abs(got[k] - ref[k]) <= 1e-12 * S[k]), (d, k)


def test_autograd_stacked_tensor_and_float32():
    n = 4096
    U = _field(n)
    Gc = synth.cotangent(n)
    Ut = torch.from_numpy(np.stack(U)).to(DEV).float().requires_grad_()
    F = autograd.flux(Ut, 0)
    assert F.shape == (5, n)
    (F * torch.from_numpy(np.stack(Gc)).to(DEV).float()).sum().backward()
    Uq = [u.astype(np.float32).astype(np.float64) for u in U]
    Gq = [g.astype(np.float32).astype(np.float64) for g in Gc]
    ref, S = oracle.flux_vjp(3, 0, G_, Uq, Gq, scale=True)
    got = Ut.grad.double().cpu().numpy()
    for k in range(5):
        assert np.all(np.abs(got[k] - ref[k]) <= 2.0 ** -24 * np.abs(ref[k]) + 64 * 2.0 ** -24 * S[k])


def test_vjp_against_central_differences():
    """<G, (F(U + h e_k) - F(U - h e_k)) / 2h> on 4,096 sampled points."""
    n = 1 << 16
    U = _field(n, seed=4)
    Gc = synth.cotangent(n)
    rng = np.random.default_rng(1)
    idx = np.sort(rng.choice(n, 4096, replace=False))
    Us = [u[idx] for u in U]
    Gs = [g[idx] for g in Gc]
    Ud, Gd = _dev(Us), _dev(Gs)
    gU = [t.cpu().numpy() for t in blocks.flux_vjp(Ud, Gd, 0, G_)]
    for k in range(5):
        h = 1e-6 * np.maximum(1.0, np.abs(Us[k]))
        Up = [u.copy() for u in Us]
        Um = [u.copy() for u in Us]
        Up[k] += h
        Um[k] -= h
        Fp = [t.cpu().numpy() for t in blocks.flux(_dev(Up), 0, G_)]
        Fm = [t.cpu().numpy() for t in blocks.flux(_dev(Um), 0, G_)]
        fd = sum((fp - fm) * g for fp, fm, g in zip(Fp, Fm, Gs)) / (2 * h)
        A = np.stack(oracle.flux_jac(3, 0, G_, Us), -1).reshape(-1, 5, 5)
        scale = (np.abs(A).sum(axis=1) * np.abs(np.stack(Gs, -1))).sum(axis=1) + 1.0
        assert np.all(np.abs(fd - gU[k]) <= 1e-7 * scale), k


@pytest.mark.slow
@pytest.mark.parametrize("dtype,dw", [(torch.float64, False), (torch.float64, True), (torch.float32, False)],
                         ids=["f64", "f64dw", "f32"])
def test_vjp_full_size_everywhere(dtype, dw):
    """N = 2^24: gU = A_x^T G at every point against the oracle."""
    n = 1 << 24
    U = _field(n)
    Gc = synth.cotangent(n)
    Ud = [torch.from_numpy(u).to(DEV).to(dtype) for u in U]
    Gd = [torch.from_numpy(g).to(DEV).to(dtype) for g in Gc]
    gU = [t.double().cpu().numpy() for t in blocks.flux_vjp(Ud, Gd, 0, G_, dw=dw)]
    Uq = [t.double().cpu().numpy() for t in Ud]
    Gq = [t.double().cpu().numpy() for t in Gd]
    del Ud, Gd
    ref, S = oracle.flux_vjp(3, 0, G_, Uq, Gq, scale=True)
    if dtype == torch.float64:
        bound = [1e-12 * s for s in S]
    else:
        bound = [2.0 ** -24 * np.abs(r) + 64 * 2.0 ** -24 * s for r, s in zip(ref, S)]
    for k in range(5):
        assert np.all(np.abs(gU[k] - ref[k]) <= bound[k]), k


@pytest.mark.parametrize("dw", [False, True], ids=["f64", "f64dw"])
@pytest.mark.parametrize("eos", [synth.EOS_NASG, synth.EOS_VDW], ids=["nasg", "vdw"])
def test_autograd_under_a_general_eos(eos, dw):
    """The differentiable flux under a general EOS: gradients equal A_d(U)^T G
    of the general-EOS oracle (1e-12 * S) and central differences of the GPU
    flux."""
    n, D = 3001, 3
    U = oracle.eos_cons_from_prim(eos, D, synth.euler_eos(n, D, seed=31))
    Gc = synth.cotangent(n, D + 2, seed=32)
    for d in range(D):
        Ud = [u.requires_grad_() for u in _dev(U)]
        F = autograd.flux(Ud, d, eos=eos, dw=dw)
        sum((f * g).sum() for f, g in zip(F, _dev(Gc))).backward()
        got = [u.grad.cpu().numpy() for u in Ud]
        ref, S = oracle.eos_flux_vjp(eos, D, d, U, Gc, scale=True)
        for k in range(D + 2):
            assert np.all(np.abs(got[k] - ref[k]) <= 1e-12 * S[k]), (d, k)
    # central differences of the GPU flux along U component j, on all points
    Ud = _dev(U)
    Gd = _dev(Gc)
    for j in range(D + 2):
        h = 1e-6 * torch.clamp(Ud[j].abs(), min=1.0)
        Up = [u.clone() for u in Ud]
        Um = [u.clone() for u in Ud]
        Up[j] += h
        Um[j] -= h
        Fp = blocks.flux_eos(Up, eos, 0, dw=dw)
        Fm = blocks.flux_eos(Um, eos, 0, dw=dw)
        fd = sum(((a - b) / (2 * h)) * g for a, b, g in zip(Fp, Fm, Gd))
        Ur = [u.clone().requires_grad_() for u in Ud]
        sum((f * g).sum() for f, g in zip(autograd.flux(Ur, 0, eos=eos, dw=dw), Gd)).backward()
        err = (fd - Ur[j].grad).abs().max().item()
        assert err <= 1e-6 * (1.0 + Ur[j].grad.abs().max().item()), j
