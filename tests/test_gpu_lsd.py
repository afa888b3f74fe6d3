"""GPU parity of the local orbitals and local Slater determinants
(swr_lsd_build through the C ABI) against the FP64 oracle
(oracle/lsd_oracle.py, Sec. 3.2, Eq. BARPOT, Eq. LSD, Appendix A, Table 1).

Both sides solve the same generalised eigenproblems in bases whose overlap
condition number is about 1e4 (LAPACK's sygvd on the host, Cholesky and
parallel Jacobi on the device), so orbital energies agree to ~1e-12, the
coefficients to ~1e-10; every integral is compared at 1e-10 of its largest
magnitude, the determinant selection exactly.
"""
import numpy as np
import pytest

from oracle import lsd_oracle as Lo

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1710_02401_gb300 import build as B
    B.build()
    from paper_1710_02401_gb300 import swr as S_
    return S_


CASES = {
    # the paper's Test 1 geometry ((-8, 8), L = 5, eps = 0.32, two nuclei at +-0.5),
    # smaller bases: 6 orbitals per subdomain, 10 determinants per subdomain
    "test1-geometry": dict(M=6, K=10, kd=30),
    # the paper's Test 1 sizes: K = 45 determinants per subdomain, 10 orbitals per
    # 1-D subdomain (a diagonal subdomain has exactly C(10, 2) = 45)
    "test1-full": dict(M=10, K=45, kd=40),
    # three subdomains, asymmetric nuclei, uneven sizes
    "small": dict(box=(-4.5, 4.5), L=3, overlap=0.3, nuclei=((-0.7, 1.0), (0.9, 2.0)), M=5, K=8, kd=24, panel=0.25,
                  q_p=10, xb_factor=0.55),
    # harmonic well, no nuclei: levels n + 1/2 in the centre subdomain
    "harmonic": dict(box=(-6.0, 6.0), L=3, overlap=0.4, nuclei=(), harmonic=1.0, M=6, K=12, kd=64,
                     xb_factor=7.0 / 4.4, ee_coef=0.5),
}


def _oracle(kw):
    p = Lo.LsdProblem(**kw)
    orbs = Lo.all_orbitals(p)
    oe = Lo.one_electron(p, orbs)
    blocks = {}
    for j in range(p.L):
        for i in range(p.L):
            pairs, Sm, Hm = Lo.lsd_hamiltonian(p, orbs, oe, i, j)
            Gn = Lo.lsd_gram(p, oe, pairs, (i, j), Lo.lsd_pairs(p, orbs, i + 1, j), (i + 1, j)) if i + 1 < p.L else None
            blocks[i + p.L * j] = (pairs, Sm, Hm, Gn)
    return p, orbs, oe, blocks


@pytest.mark.parametrize("name", list(CASES))
def test_lsd_build_matches_the_oracle(S, name):
    kw = CASES[name]
    p, orbs, oe, blocks = _oracle(kw)
    g = S.lsd_build(**kw)
    lam = np.array([o.lam for o in orbs])
    np.testing.assert_allclose(g["lam"], lam, rtol=0, atol=1e-10 * max(1.0, np.abs(lam).max()))
    coef = np.array([o.coef for o in orbs])
    np.testing.assert_allclose(g["coef"], coef, rtol=0, atol=1e-8 * np.abs(coef).max())
    for key in ("S1", "h1", "J1"):
        ref = getattr(oe, key.rstrip("1"))
        np.testing.assert_allclose(g[key], ref, rtol=0, atol=1e-10 * np.abs(ref).max(), err_msg=key)
    hmax = max(np.abs(b[2]).max() for b in blocks.values())
    for om, (pairs, Sm, Hm, Gn) in blocks.items():
        assert [tuple(x) for x in g["pairs"][om]] == pairs, om
        np.testing.assert_allclose(g["S_lsd"][om], Sm, rtol=0, atol=1e-10, err_msg=f"S {om}")
        np.testing.assert_allclose(g["H_lsd"][om], Hm, rtol=0, atol=1e-10 * hmax, err_msg=f"H {om}")
        if Gn is not None:
            np.testing.assert_allclose(g["G_next"][om], Gn, rtol=0, atol=1e-10, err_msg=f"G {om}")
        else:
            assert not np.any(g["G_next"][om])
    if name == "harmonic":
        np.testing.assert_allclose(g["lam"][1], np.arange(6) + 0.5, atol=1e-8)
    if name.startswith("test1"):
        # Table 1's structure: the central subdomain's determinants orthonormal,
        # their inner products with the neighbour's (x1 in D_4) small
        c = 2 + 5 * 2
        np.testing.assert_allclose(g["S_lsd"][c][:4, :4], np.eye(4), atol=1e-13)
        assert 1e-8 < np.abs(g["G_next"][c][:4, :2]).max() < 0.1
        print(f"\n[{name}] Table 1 (GPU): <v_i, v_j> off-diagonal max "
              f"{np.abs(g['S_lsd'][c][:4, :4] - np.eye(4)).max():.1e}; <v_i, w_j> =\n{g['G_next'][c][:4, :2]}")


def test_lsd_build_rejects_invalid_problems(S):
    with pytest.raises(S.SWRError) as e:
        S.lsd_build(M=4, K=7, kd=20)  # a diagonal subdomain has only M (M - 1) / 2 = 6 determinants
    assert e.value.status == S.SWR_EINVAL
    with pytest.raises(S.SWRError) as e:
        S.lsd_build(kd=65)
    assert e.value.status == S.SWR_EINVAL
