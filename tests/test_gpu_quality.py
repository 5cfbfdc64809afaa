"""The library against the paper's quality claims (Figures 3, 5-7 and 9-10) on
Matrices 1-3 of Section 7, through the C ABI, in the FP64 and FP64-emulation
modes: the same checks as the oracle's (tests/_quality.py), on the GPU's
factorizations and RSVD.  Run with -s to print the summary table."""
import numpy as np
import pytest

from paper_1812_06007_gb300 import workloads as W

from ._quality import check_lemma, check_quality

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_1812_06007_gb300 import binding, build
    build.build()
    return binding


def _dev(x):
    import torch
    from paper_1812_06007_gb300.binding import as_colmajor
    return as_colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def _host(t):
    import torch
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("mode", ["fp64", "fp64emu"])
def test_gpu_quality_claims(B, mode):
    md = {"fp64": B.PURL_MODE_FP64, "fp64emu": B.PURL_MODE_FP64_EMU}[mode]
    rows = []
    for name in ("fast", "slow", "s"):
        A = W.quality_matrix_np(name)
        reorth = name != "slow"
        facts = {q: tuple(_host(x) for x in B.purl_urv_factor(_dev(A), q, reorth, W.SEED_G, mode=md))
                 for q in (0, 1, 2)}
        rows += check_quality(name, A, facts)
    print(f"\n[{mode}] matrix q  median ||A-A_k||/sigma_k+1  max  median sigma_k(R11)/sigma_k")
    for name, q, med, mx, r11 in rows:
        print(f"[{mode}] {name:5s} {q}  {med:.3f}  {mx:.2f}  {r11:.3f}")


@pytest.mark.parametrize("q", [0, 1])
def test_gpu_lemma_rsvd_vs_powerurv(B, q):
    A = W.quality_matrix_np("slow")
    U, R, V = (_host(x) for x in B.purl_urv_factor(_dev(A), q, False, W.SEED_G))
    Ur, S, Vr = (_host(x) for x in B.purl_rsvd(_dev(A), l=60, q=q, seed=W.SEED_G, reorth=False))
    eu, er, ru, rv = check_lemma(A, U, V, Ur, Vr, 60)
    print(f"\n[lemma q={q}] ||A-U_l U_l^T A|| = {eu:.6e}, RSVD {er:.6e}; median over k <= 30 of "
          f"PowerURV/RSVD: U {ru:.2f}, V {rv:.2f}")
