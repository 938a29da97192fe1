"""Plain MPS circuit evolution with truncated pivoted-QR splitting (test infrastructure).

ORACLE — slow, obviously correct, complex128.  Only tests, the package smoke
check and the benchmark's CPU-baseline leg use it; the GPU library never calls
it.  Every step follows the paper's description:

* State (Sec. II-B.1, Sec. III-A.1): n sites, site i a row-major complex array
  (chi_i, 2, chi_{i+1}) with chi_0 = chi_n = 1; |0...0> has every site
  [1, 0] of shape (1, 2, 1).
* One-qubit gate (Sec. II-A.2, tensor application Sec. III-C.2):
  A[l, s, r] <- sum_s' u[s, s'] A[l, s', r].
* Two-qubit gate on (i, i+1) (Sec. III-C.2): contract the two sites over the
  shared bond (Sec. III-B.1), contract the gate into the physical indices,
  theta[l, a, b, r] = sum_{cd} g[2a+b, 2c+d] X[l, c, d, r], read theta as the
  (2 chi_l) x (2 chi_r) matrix with row (l, a) and column (b, r), and split it
  by the truncated column-pivoted QR theta P = Q R (Sec. III-B.2, QR with
  pivoting) stopped after k = min(2 chi_l, 2 chi_r, chi_max) pivots:
  the left site becomes Q[:, :k] reshaped (chi_l, 2, k) and the right site
  R[:k, :] P^T reshaped (k, 2, chi_r).  The state is never renormalised, so
  its squared norm is the norm fidelity of Sec. III-E.  With truncation="svd"
  the split is the truncated SVD instead (Sec. III-B.2 Table III, compared with
  pivoted QR in Sec. IV-A.1; oracle/svd.py): left site U[:, :k], right site
  diag(S[:k]) V^dagger[:k, :], same k.  With truncation="rqrcp" the pivots are
  chosen on a random sketch (oracle/rqrcp.py; one of the QR improvements the
  bond-truncation discussion of Sec. IV-A.1 points to), the split is otherwise the
  same; two-site split number s uses the sketch seed sketch_seed + s.
* SWAP (Sec. III-C.4): the two-qubit path with the SWAP gate; a gate on
  non-adjacent positions lo < hi moves the qubit at lo rightwards by SWAPs on
  bonds (lo, lo+1) ... (hi-2, hi-1), applies the gate on (hi-1, hi), then
  SWAPs back in reverse order.
* Orthogonality centre (Sec. III-C.1): under the "canon" policy the centre is
  moved to site i before a gate on (i, i+1) by plain QR (rightward move: the Q
  factor stays, R is multiplied into the next site) or LQ (leftward move, as QR
  of the conjugate transpose; L is multiplied into the previous site), without
  truncation; after the gate the centre is site i+1.  The "local" policy never
  moves the centre.
* MPO application (Sec. III-C.3, zip-up): an operator W_first ... W_last with
  tensors W[a, b, out, in] (a = 1 on the first, b = 1 on the last) is contracted
  into the sites left to right: with the carried matrix C[kk, a, l] (identity at
  the start), Z[kk, out, b, r] = sum W[a, b, out, in] C[kk, a, l] A[l, in, r];
  Z as the (2 kk) x (b r) matrix is split by the truncated pivoted QR, Q becomes
  the site and R P^T the next carried C; the last Z is the last site.  The new
  bond is capped at min(chi_max, 2 cap) with cap = min(2^b, 2^(n-b), chi_max),
  the chain's physical bound, so one MPO of bond 2 never truncates for lack of
  room; afterwards every bond of the range above its physical bound is brought
  back to it by a split of the identity two-site gate, right to left (exact
  under the canonical policy, where the cut's Schmidt rank is at most cap).
* Amplitude: <x|psi> = A_0[:, x_0, :] A_1[:, x_1, :] ... (1x1 product).
* Norm fidelity (Sec. III-E): F = <psi|psi> by transfer matrices
  E <- sum_s A[:, s, :]^H E A[:, s, :].
"""

import numpy as np

from . import qr as _qr
from . import rqrcp as _rqrcp
from . import svd as _svd


def _swap_gate():
    g = np.zeros((4, 4), dtype=np.complex128)
    for a in range(2):
        for b in range(2):
            g[2 * b + a, 2 * a + b] = 1.0
    return g


SWAP = _swap_gate()
IDENTITY4 = np.eye(4, dtype=np.complex128)


def physical_bond(n, b, chi):
    """Largest Schmidt rank across cut b of an n-qubit chain, capped at chi."""
    e = min(b, n - b)
    return chi if e >= 30 else min(2**e, chi)


class OracleMPS:
    def __init__(self, n, chi_max, policy="canon", truncation="qrcp", sketch_seed=0):
        assert n >= 1 and chi_max >= 1 and policy in ("canon", "local")
        assert truncation in ("qrcp", "svd", "rqrcp")
        self.n = n
        self.chi_max = chi_max
        self.policy = policy
        self.truncation = truncation
        self.sketch_seed = sketch_seed  # rqrcp: split number s uses seed sketch_seed + s
        self.sites = []
        for _ in range(n):
            s = np.zeros((1, 2, 1), dtype=np.complex128)
            s[0, 0, 0] = 1.0
            self.sites.append(s)
        self.centre = 0
        self.discarded = []  # discarded weight of every two-qubit split, in order
        self.n_two_site = 0

    # ---- state access -------------------------------------------------
    def bond_dims(self):
        return [1] + [s.shape[2] for s in self.sites]

    def set_sites(self, sites, centre=0):
        assert len(sites) == self.n
        for i in range(self.n - 1):
            assert sites[i].shape[2] == sites[i + 1].shape[0]
        self.sites = [np.array(s, dtype=np.complex128, copy=True) for s in sites]
        self.centre = centre

    def copy(self):
        o = OracleMPS(self.n, self.chi_max, self.policy, self.truncation, self.sketch_seed)
        o.sites = [s.copy() for s in self.sites]
        o.centre = self.centre
        o.discarded = list(self.discarded)
        o.n_two_site = self.n_two_site
        return o

    # ---- gates -------------------------------------------------------
    def apply_1q(self, q, u):
        u = np.asarray(u, dtype=np.complex128)
        self.sites[q] = np.einsum("ab,lbr->lar", u, self.sites[q])

    def _move_right(self, j):
        a = self.sites[j]
        cl, _, cr = a.shape
        q, r, _, _ = _qr.cpqr(a.reshape(2 * cl, cr), pivot=False)
        k = q.shape[1]
        self.sites[j] = np.ascontiguousarray(q).reshape(cl, 2, k)
        nxt = self.sites[j + 1]
        self.sites[j + 1] = (r @ nxt.reshape(cr, -1)).reshape(k, 2, nxt.shape[2])

    def _move_left(self, j):
        a = self.sites[j]
        cl, _, cr = a.shape
        m = a.reshape(cl, 2 * cr)
        q, r, _, _ = _qr.cpqr(m.conj().T, pivot=False)  # m^H = q r  ->  m = r^H q^H
        k = q.shape[1]
        self.sites[j] = np.ascontiguousarray(q.conj().T).reshape(k, 2, cr)
        prv = self.sites[j - 1]
        self.sites[j - 1] = (prv.reshape(-1, cl) @ r.conj().T).reshape(prv.shape[0], 2, k)

    def move_centre(self, target):
        while self.centre < target:
            self._move_right(self.centre)
            self.centre += 1
        while self.centre > target:
            self._move_left(self.centre)
            self.centre -= 1

    def apply_2q(self, i, g, chi_max=None):
        """Gate g on adjacent sites (i, i+1); returns the discarded weight."""
        chi = self.chi_max if chi_max is None else min(chi_max, self.chi_max)
        if self.policy == "canon":
            self.move_centre(i)
        g = np.asarray(g, dtype=np.complex128).reshape(2, 2, 2, 2)
        a, b = self.sites[i], self.sites[i + 1]
        cl, cm, cr = a.shape[0], a.shape[2], b.shape[2]
        x = (a.reshape(2 * cl, cm) @ b.reshape(cm, 2 * cr)).reshape(cl, 2, 2, cr)
        theta = np.einsum("abcd,lcdr->labr", g, x).reshape(2 * cl, 2 * cr)
        if self.truncation == "svd":
            q, right, _, disc = _svd.svd_split(theta, chi)
            k = q.shape[1]
        elif self.truncation == "rqrcp":
            res = _rqrcp.rqrcp(theta, chi, seed=self.sketch_seed + self.n_two_site)
            q, k, disc = res["q"], res["k"], res["discarded"]
            right = np.zeros((k, 2 * cr), dtype=np.complex128)
            right[:, res["jpvt"]] = res["r"]
        else:
            q, r, jpvt, disc = _qr.cpqr(theta, kmax=chi, pivot=True)
            k = q.shape[1]
            right = np.zeros((k, 2 * cr), dtype=np.complex128)
            right[:, jpvt] = r
        self.sites[i] = np.ascontiguousarray(q).reshape(cl, 2, k)
        self.sites[i + 1] = right.reshape(k, 2, cr)
        if self.policy == "canon":
            self.centre = i + 1
        self.discarded.append(disc)
        self.n_two_site += 1
        return disc

    def apply_mpo(self, first, ws, chi_max=None):
        """Zip-up application of the MPO ``ws`` (list of W[a, b, out, in]) to the sites
        first .. first+len(ws)-1; returns the discarded weights of its splits."""
        chi = self.chi_max if chi_max is None else min(chi_max, self.chi_max)
        ws = [np.asarray(w, dtype=np.complex128) for w in ws]
        last = first + len(ws) - 1
        assert ws[0].shape[0] == 1 and ws[-1].shape[1] == 1
        if len(ws) == 1:
            self.apply_1q(first, ws[0][0, 0])
            return []
        if self.policy == "canon":
            self.move_centre(first)
        n = self.n
        discs = []
        cl = self.sites[first].shape[0]
        c = np.eye(cl, dtype=np.complex128).reshape(cl, 1, cl)  # C[kk, a, l]
        for j, w in enumerate(ws):
            i = first + j
            y = np.einsum("kal,lsr->kasr", c, self.sites[i])
            z = np.einsum("abts,kasr->ktbr", w, y)
            kk, _, bd, cr = z.shape
            if i == last:
                self.sites[i] = np.ascontiguousarray(z.reshape(kk, 2, cr))
                break
            cap = min(chi, 2 * physical_bond(n, i + 1, chi))
            q, r, jpvt, disc = _qr.cpqr(z.reshape(2 * kk, bd * cr), kmax=cap, pivot=True)
            k = q.shape[1]
            right = np.zeros((k, bd * cr), dtype=np.complex128)
            right[:, jpvt] = r
            self.sites[i] = np.ascontiguousarray(q).reshape(kk, 2, k)
            c = right.reshape(k, bd, cr)
            self.discarded.append(disc)
            self.n_two_site += 1
            discs.append(disc)
        if self.policy == "canon":
            self.centre = last
        for b in range(last, first, -1):
            cap = physical_bond(n, b, chi)
            if self.sites[b].shape[0] > cap:
                discs.append(self.apply_2q(b - 1, IDENTITY4, cap))
        return discs

    def swap(self, i, chi_max=None):
        return self.apply_2q(i, SWAP, chi_max)

    def apply_2q_routed(self, q1, q2, g, chi_max=None):
        """Gate g on the ordered pair (q1, q2), routed by SWAP chains if needed."""
        g = np.asarray(g, dtype=np.complex128)
        assert q1 != q2
        if q1 > q2:
            q1, q2 = q2, q1
            g = SWAP @ g @ SWAP
        for b in range(q1, q2 - 1):
            self.swap(b, chi_max)
        self.apply_2q(q2 - 1, g, chi_max)
        for b in range(q2 - 2, q1 - 1, -1):
            self.swap(b, chi_max)

    def permute(self, order, chi_max=None):
        """Site permutation by nearest-neighbour SWAPs, bubble-sort order (Sec. III-C,
        "Site permutation"; the RCS re-embedding of Sec. III-D.2): afterwards chain
        position p holds the site that was at position order[p].  Each pass walks the
        chain left to right and swaps neighbours whose target positions are out of
        order, updating the tuple of target positions as it goes.  Returns the
        number of SWAPs (the number of inversions of the permutation)."""
        n = len(self.sites)
        order = [int(x) for x in order]
        assert sorted(order) == list(range(n)), "order must be a permutation of the positions"
        dest = [0] * n  # dest[q] = final position of the site now at q
        for p, q in enumerate(order):
            dest[q] = p
        swaps = 0
        changed = True
        while changed:
            changed = False
            for q in range(n - 1):
                if dest[q] > dest[q + 1]:
                    self.swap(q, chi_max)
                    dest[q], dest[q + 1] = dest[q + 1], dest[q]
                    swaps += 1
                    changed = True
        return swaps

    def permute_layers(self, order, chi_max=None):
        """The same site permutation by odd-even transposition sort, the parallel form of
        the bubble sort above: pass t looks at the pairs (q, q+1) with q of the parity of
        t, left to right, and swaps every pair whose target positions are out of order;
        the SWAPs of one pass act on disjoint bonds, so they form one circuit layer.
        Passes alternate until an even and an odd pass in a row find nothing to swap.
        Returns (SWAPs, passes that swapped); the SWAP count is again the number of
        inversions of the permutation."""
        n = len(self.sites)
        order = [int(x) for x in order]
        assert sorted(order) == list(range(n)), "order must be a permutation of the positions"
        dest = [0] * n
        for p, q in enumerate(order):
            dest[q] = p
        swaps = passes = idle = 0
        parity = 0
        while idle < 2:
            layer = []
            for q in range(parity, n - 1, 2):
                if dest[q] > dest[q + 1]:
                    layer.append(q)
                    dest[q], dest[q + 1] = dest[q + 1], dest[q]
            for q in layer:
                self.swap(q, chi_max)
            swaps += len(layer)
            passes += 1 if layer else 0
            idle = 0 if layer else idle + 1
            parity ^= 1
        return swaps, passes

    def run(self, ops, chi_max=None):
        for op in ops:
            if op[0] == "1q":
                self.apply_1q(op[1], op[2])
            elif op[0] == "perm":
                self.permute(op[1], chi_max)
            elif op[0] == "mpo":
                self.apply_mpo(op[1], op[2], chi_max)
            else:
                self.apply_2q_routed(op[1], op[2], op[3], chi_max)

    # ---- observables -------------------------------------------------
    def amplitude(self, bits):
        v = np.ones((1, 1), dtype=np.complex128)
        for i in range(self.n):
            v = v @ self.sites[i][:, int(bits[i]), :]
        return complex(v[0, 0])

    def overlap(self, other):
        """<self|other> by transfer matrices."""
        e = np.ones((1, 1), dtype=np.complex128)
        for a, b in zip(self.sites, other.sites):
            e = sum(a[:, s, :].conj().T @ e @ b[:, s, :] for s in range(2))
        return complex(e[0, 0])

    def norm2(self):
        """Norm fidelity <psi|psi> (Sec. III-E)."""
        return self.overlap(self).real

    def centre_norm2(self):
        return float(np.vdot(self.sites[self.centre], self.sites[self.centre]).real)

    def statevector(self):
        """Dense 2^n vector (small n only); index bit n-1-i is site i."""
        v = self.sites[0].reshape(2, -1)
        for i in range(1, self.n):
            s = self.sites[i]
            v = (v @ s.reshape(s.shape[0], -1)).reshape(-1, s.shape[2])
        return v.reshape(-1)
