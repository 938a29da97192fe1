"""Full-size checks at the bond dimension of the headline workload (chi = 4096,
theta 8192 x 8192), in the launch configuration the benchmark times: one gate and
one left centre move through the C ABI, verified by properties that hold at any size
and by what a brute-force computation can give column by column.  The reference
arithmetic here is PyTorch (FP64) on the GPU; the oracle cannot factor an
8192 x 8192 matrix in test time.

Properties (Sec. III-B.2 pivoted QR, Sec. III-C.2 split, Sec. III-E fidelity):
  * the new left site Q (8192 x 4096) has orthonormal columns;
  * the new right site equals Q^H theta on sampled columns (R P^T is the projection
    of theta onto the kept subspace), theta computed independently from the input
    sites and the gate;
  * ||R P^T||^2 + discarded weight = ||theta||^2;
  * the first pivot is the column of theta with the largest norm, and |R_00| is that norm;
  * a left centre move keeps the two-site block and leaves the right site with
    orthonormal rows.
"""

import numpy as np
import pytest

from workloads import gates

pytestmark = pytest.mark.gpu

CHI = 4096


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__

    __graft_entry__.build()


# Bars: typical rounding at these sizes is u * sqrt(8192) (u = 6e-8 for the FP32 bulk of
# the mixed path, 1.1e-16 for FP64): 5e-6 and 1e-14.  The bars leave a margin of ~20 (mixed)
# and ~100 (FP64) over that: orthonormality `orth` (absolute, per element), the projection
# and the two-site block `proj` (relative to the largest |theta|), the norm identity and
# the first pivot `rel` (relative).
BARS = {"mixed": {"orth": 1e-4, "proj": 1e-4, "rel": 1e-5},
        "fp64": {"orth": 1e-12, "proj": 1e-11, "rel": 1e-12}}


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_full_size_gate_and_centre_move(prec):
    import torch

    from paper_2505_06119_gb300 import MPS

    torch.backends.cuda.matmul.allow_tf32 = False
    bar = BARS[prec]
    dev = torch.device("cuda:0")
    chi = CHI
    n, i = 28, 13  # bonds i, i+1, i+2 reserve chi
    rng = np.random.default_rng(20250509)
    dt = np.complex64 if prec == "mixed" else np.complex128

    def site():
        x = rng.standard_normal((chi, 2, chi)) + 1j * rng.standard_normal((chi, 2, chi))
        return (x / np.linalg.norm(x)).astype(dt)

    a, b = site(), site()
    g = gates.haar_unitary(rng, 4)
    with MPS(n, chi, precision=prec, policy="local") as m:
        m.set_site(i, a)
        m.set_site(i + 1, b)
        # theta = gate applied to A_i A_{i+1}, rows (l, a), columns (b, r), in FP64
        A = torch.from_numpy(a.reshape(2 * chi, chi)).to(dev, torch.complex128)
        B = torch.from_numpy(b.reshape(chi, 2 * chi)).to(dev, torch.complex128)
        X = (A @ B).reshape(chi, 2, 2, chi)
        G = torch.from_numpy(np.ascontiguousarray(g.reshape(2, 2, 2, 2))).to(dev, torch.complex128)
        theta = torch.einsum("abcd,lcdr->labr", G, X).reshape(2 * chi, 2 * chi)
        del A, B, X
        d0 = m.discarded()[0]
        m.apply_2q(i, g)
        disc = m.discarded()[0] - d0
        assert m.bond_dims()[i + 1] == chi
        Q = torch.from_numpy(m.get_site(i)).to(dev).reshape(2 * chi, chi)
        RP = torch.from_numpy(m.get_site(i + 1)).to(dev).reshape(chi, 2 * chi)
        scale = theta.abs().max().item()
        # orthonormal Q
        eye = torch.eye(chi, dtype=torch.complex128, device=dev)
        assert (Q.conj().T @ Q - eye).abs().max().item() < bar["orth"]
        # R P^T = Q^H theta on sampled columns
        cols = torch.from_numpy(rng.choice(2 * chi, 512, replace=False)).to(dev)
        proj = Q.conj().T @ theta[:, cols]
        assert (RP[:, cols] - proj).abs().max().item() < bar["proj"] * scale
        # norm identity (Sec. III-E): kept + discarded = total
        tot = (theta.abs() ** 2).sum().item()
        kept = (RP.abs() ** 2).sum().item()
        assert abs(kept + disc - tot) < bar["rel"] * tot
        # first pivot = largest column norm of theta, |R_00| = that norm
        cn = (theta.abs() ** 2).sum(0).sqrt()
        p0 = int(torch.argmax(cn).item())
        assert abs(RP[0, p0].abs().item() - cn[p0].item()) < bar["rel"] * cn[p0].item()
        # left centre move: LQ of site i+1, L absorbed into site i
        block = Q @ RP[:, cols]
        m.set_centre(i + 1)
        m.move_centre(i)
        A2 = torch.from_numpy(m.get_site(i)).to(dev).reshape(2 * chi, chi)
        B2 = torch.from_numpy(m.get_site(i + 1)).to(dev).reshape(chi, 2 * chi)
        assert (B2 @ B2.conj().T - eye).abs().max().item() < bar["orth"]
        assert (A2 @ B2[:, cols] - block).abs().max().item() < bar["proj"] * scale
