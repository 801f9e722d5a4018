"""The MPDO noisy-circuit simulator of Sec. II.C-II.D, FP64 NumPy.  Test infrastructure only.

State: one rank-4 tensor per qubit, T[l, p, n, r] (left bond, physical, Kraus
leg, right bond), Sec. II.C.  The represented density matrix is
rho = sum_{n_0..n_{N-1}} |psi_n><psi_n| with psi_n[p_0..p_{N-1}] the matrix
product T_0[:, p_0, n_0, :] ... T_{N-1}[:, p_{N-1}, n_{N-1}, :], which is the
open-chain trace of the local densities M = sum_n T T* of Sec. II.C.

Steps, in the paper's order:
  * a noisy gate is K_i = N_i U (Eq. for K_i in Sec. II.C; noise after the gate);
    its Kraus index becomes a new leg joined to the site's Kraus leg (Fig. 2b,c);
    for a two-qubit gate the new leg joins the right site q+1, for a three-qubit channel site q+2;
  * bond truncation (Fig. 3b): the chain is kept in canonical form by QR sweeps
    and the two-site tensor is split by an SVD that keeps the top chi_max values;
  * Kraus-leg truncation (Eq. svdNoise, Fig. 3a): the site tensor as a
    (p, l, r) x n matrix is SVD-truncated to kappa_max values, T' = U S (= T V).
  * the paper's global schedule (Sec. II.D): QR decompositions from left to right into canonical
    form, then an SVD truncation of every bond from right to left (truncate_bonds, run where a
    circuit places a SWEEP op).
Readings where the paper is silent: truncation runs per gate with the
orthogonality centre on the touched site (either site of a two-qubit gate); after a two-qubit gate the bond is
split first and the right site's Kraus leg truncated second (trunc_order "split_first"; the order
"kraus_first" truncates the merged tensor's new Kraus leg before the split); nothing is
renormalised and every readout is divided by Tr(rho); singular values at or
below tol * sigma_max are dropped as numerically zero.

Pinned by tests/test_oracle_mpdo.py against the dense simulator (no truncation,
1e-12), the Eckart-Young identity of Sec. II.D and the exactness of the
decomposition when the caps are at least the ranks.
"""
from __future__ import annotations

import numpy as np

from .channels import chi_to_kraus


class MPDO:
    def __init__(self, n: int, chi_max: int, kappa_max: int, tol: float = 1e-13,
                 auto_truncate: bool = True, trunc_order: str = "split_first"):
        if trunc_order not in ("split_first", "kraus_first"):
            raise ValueError(trunc_order)
        self.trunc_order = trunc_order
        self.n = n
        self.chi_max = chi_max
        self.kappa_max = kappa_max
        self.tol = tol
        self.auto_truncate = auto_truncate
        site = np.zeros((1, 2, 1, 1), dtype=np.complex128)
        site[0, 0, 0, 0] = 1.0
        self.sites = [site.copy() for _ in range(n)]
        self.centre = 0
        self.discarded_chi = 0.0
        self.discarded_kappa = 0.0
        self.min_gap = np.inf   # smallest (s_k^2 - s_{k+1}^2)/s_1^2 over truncations that cut
        self.cuts = []          # (relative gap, kept count, s^2 of every truncation that cuts)
        self.log = []           # (kind, site, kept, available, discarded weight)
        # optional (eps, rng): every matrix about to be SVD-truncated is perturbed by eps * max|entry|
        # complex Gaussian noise first (models rounding; used only to pin cut_allowance)
        self.perturb = None

    # ------------------------------------------------------------ canonical form
    def _shift_right(self, q: int) -> None:
        A = self.sites[q]
        dl, _, dn, dr = A.shape
        Q, R = np.linalg.qr(A.reshape(dl * 2 * dn, dr))
        self.sites[q] = Q.reshape(dl, 2, dn, Q.shape[1])
        self.sites[q + 1] = np.einsum("xb,bpnr->xpnr", R, self.sites[q + 1])

    def _shift_left(self, q: int) -> None:
        A = self.sites[q]
        dl, _, dn, dr = A.shape
        Q, R = np.linalg.qr(A.reshape(dl, 2 * dn * dr).conj().T)  # A = R^dag Q^dag
        self.sites[q] = Q.conj().T.reshape(Q.shape[1], 2, dn, dr)
        self.sites[q - 1] = np.einsum("lpnb,bx->lpnx", self.sites[q - 1], R.conj().T)

    def move_centre(self, q: int) -> None:
        """QR sweeps that leave every site left of q left-isometric and right of q right-isometric."""
        while self.centre < q:
            self._shift_right(self.centre)
            self.centre += 1
        while self.centre > q:
            self._shift_left(self.centre)
            self.centre -= 1

    # ------------------------------------------------------------ truncation
    def _keep(self, s: np.ndarray, cap: int):
        """How many singular values to keep, and the discarded weight sum_{dropped} s^2 / sum s^2."""
        total = float(np.sum(s ** 2))
        if total == 0.0:
            return 1, 0.0
        nz = int(np.sum(s > self.tol * s[0]))
        k = max(1, min(cap, nz))
        dropped = float(np.sum(s[k:] ** 2)) / total
        if k < nz:
            s2 = s ** 2
            gap = float((s2[k - 1] - s2[k]) / s2[0])
            self.min_gap = min(self.min_gap, gap)
            self.cuts.append((gap, k, s2.copy()))
        return k, dropped

    def _perturbed(self, M: np.ndarray) -> np.ndarray:
        if self.perturb is None:
            return M
        eps, rng = self.perturb
        noise = rng.normal(size=M.shape) + 1j * rng.normal(size=M.shape)
        return M + (eps * np.max(np.abs(M)) / np.sqrt(2)) * noise

    def cut_allowance(self, threshold: float) -> float:
        """Allowance on a normalised readout (operator norm 1) for truncations that cut inside a
        near-degenerate cluster, where the truncation of Sec. II.D is not unique.

        A cut with relative gap (s_k^2 - s_{k+1}^2) / s_1^2 >= threshold contributes nothing.  Below
        it, the kept directions whose s_i^2 lies within threshold * s_1^2 of the first dropped one
        may be exchanged for dropped directions of the same cluster.  Exchanging directions of total
        weight W (in units of the unnormalised state, since sum s^2 = Tr rho with the centre on the
        truncated site) moves the state by at most 2 W in trace norm, and the normalisation by the
        final trace T doubles that bound for Tr(rho O) / Tr rho.  The sum over such cuts of 4 W / T is
        returned; it is 0 when every cut is separated by at least `threshold`."""
        bad = [(k, s2) for gap, k, s2 in self.cuts if gap < threshold]
        if not bad:
            return 0.0
        tf = self.trace()
        a = 0.0
        for k, s2 in bad:
            near = (s2[:k] - s2[k]) < threshold * s2[0]
            a += 4.0 * float(np.sum(s2[:k][near])) / tf
        return a

    def truncate_kraus(self, q: int, kappa: int = 0) -> float:
        """Eq. (svdNoise): T as a (p, l, r) x n matrix = U S V^dag; keep the top kappa; T' = T V."""
        cap = kappa if kappa > 0 else self.kappa_max
        self.move_centre(q)
        A = self.sites[q]
        dl, _, dn, dr = A.shape
        M = self._perturbed(A.transpose(0, 1, 3, 2).reshape(dl * 2 * dr, dn))
        _, s, Vh = np.linalg.svd(M, full_matrices=False)
        k, w = self._keep(s, cap)
        Mt = M @ Vh[:k].conj().T
        self.sites[q] = Mt.reshape(dl, 2, dr, k).transpose(0, 1, 3, 2).copy()
        self.discarded_kappa += w
        self.log.append(("kappa", q, k, len(s), w))
        return w

    def truncate_bonds(self, chi: int) -> float:
        """The global bond truncation of Sec. II.D (Fig. 3b): QR decompositions from left to right
        bring the chain into canonical form (centre on the last site), then every bond is
        SVD-truncated to chi values from right to left.  With the centre on site c, T_c as an
        l x (p, n, r) matrix = U S V^dag carries the Schmidt decomposition of bond (c-1, c);
        T_c <- V^dag[:k] and T_{c-1} <- T_{c-1} U[:, :k] S[:k] moves the centre to c-1.  Returns the
        summed discarded weight of the sweep; the centre ends on site 0."""
        self.move_centre(self.n - 1)
        total = 0.0
        for c in range(self.n - 1, 0, -1):
            A = self.sites[c]
            dl, _, dn, dr = A.shape
            Um, s, Vh = np.linalg.svd(self._perturbed(A.reshape(dl, 2 * dn * dr)), full_matrices=False)
            k, w = self._keep(s, chi)
            self.sites[c] = Vh[:k].reshape(k, 2, dn, dr)
            self.sites[c - 1] = np.einsum("lpnb,bx->lpnx", self.sites[c - 1], Um[:, :k] * s[:k])
            self.centre = c - 1
            self.discarded_chi += w
            self.log.append(("chi", c - 1, k, len(s), w))
            total += w
        return total

    # ------------------------------------------------------------ noisy gates
    def apply_1q(self, q: int, U: np.ndarray, kraus) -> None:
        """T'[l, p', (k, n), r] = sum_p (N_k U)[p', p] T[l, p, n, r]; then Kraus-leg truncation."""
        self.move_centre(q)
        K = np.stack([N @ U for N in kraus])  # [k, p', p]
        A = self.sites[q]
        dl, _, dn, dr = A.shape
        At = np.einsum("kab,lbnr->laknr", K, A)              # new leg index k * dn + n
        self.sites[q] = At.reshape(dl, 2, len(kraus) * dn, dr)
        if self.auto_truncate:
            self.truncate_kraus(q)

    def apply_2q(self, q: int, U: np.ndarray, kraus) -> None:
        """Two-site update on (q, q+1): merge, apply K_k = N_k U with a new Kraus leg on site q+1,
        split by the SVD of the (l, p1, n1) x (p2, k, n2, r) matrix keeping chi_max values, then
        truncate the Kraus leg of site q+1 ("split_first").  With trunc_order "kraus_first" the new
        Kraus leg of the merged tensor is truncated first and the bond split second.  The split only needs every site left of q
        left-isometric and every site right of q+1 right-isometric, so the centre may sit on either
        of the two sites; it is moved only when it is elsewhere."""
        if self.centre not in (q, q + 1):
            self.move_centre(q)
        A1, A2 = self.sites[q], self.sites[q + 1]
        dl, _, dn1, _ = A1.shape
        _, _, dn2, dr = A2.shape
        rk = len(kraus)
        K = np.stack([N @ U for N in kraus]).reshape(rk, 2, 2, 2, 2)  # [k, p1', p2', p1, p2]
        theta = np.einsum("lanb,bcmr->lancmr", A1, A2)                # [l, p1, n1, p2, n2, r]
        theta = np.einsum("kxyac,lancmr->lxnykmr", K, theta)          # [l, p1', n1, p2', k, n2, r]
        dk = rk * dn2
        if self.auto_truncate and self.trunc_order == "kraus_first":
            # Eq. (svdNoise) on the merged tensor first: its new Kraus leg (k, n2) against all other
            # indices (l, p1', n1, p2', r), keep kappa_max values; the bond split below then sees the
            # already truncated leg and site q+1 needs no second Kraus truncation
            M = self._perturbed(theta.reshape(dl, 2, dn1, 2, dk, dr).transpose(0, 1, 2, 3, 5, 4).reshape(-1, dk))
            _, sk, Vkh = np.linalg.svd(M, full_matrices=False)
            nu, wk = self._keep(sk, self.kappa_max)
            theta = (M @ Vkh[:nu].conj().T).reshape(dl, 2, dn1, 2, dr, nu).transpose(0, 1, 2, 3, 5, 4)
            self.discarded_kappa += wk
            self.log.append(("kappa", q + 1, nu, len(sk), wk))
            dk = nu
        mat = self._perturbed(theta.reshape(dl * 2 * dn1, 2 * dk * dr))
        Um, s, Vh = np.linalg.svd(mat, full_matrices=False)
        k, w = self._keep(s, self.chi_max)
        self.sites[q] = Um[:, :k].reshape(dl, 2, dn1, k)
        self.sites[q + 1] = (s[:k, None] * Vh[:k]).reshape(k, 2, dk, dr)
        self.centre = q + 1
        self.discarded_chi += w
        self.log.append(("chi", q, k, len(s), w))
        if self.auto_truncate and self.trunc_order == "split_first":
            self.truncate_kraus(q + 1)

    def apply_3q(self, q: int, U: np.ndarray, kraus) -> None:
        """Three-site update on (q, q+1, q+2) for a three-qubit channel, e.g. the crosstalk channel a
        tomography of a two-qubit gate and its neighbour yields (Fig. 13b): the three sites are merged,
        K_k = N_k U (8 x 8) applied with the new Kraus leg on site q+2 (the rightmost, as for two-qubit
        gates), the merged tensor split by two SVDs that keep chi_max values, first
        (l, p1', n1) | (p2', n2, p3', k, n3, r) and then (b, p2', n2) | (p3', k, n3, r), and the Kraus
        leg of site q+2 truncated to kappa_max.  The centre is moved onto q first and ends on q+2."""
        self.move_centre(q)
        A1, A2, A3 = self.sites[q], self.sites[q + 1], self.sites[q + 2]
        dl, _, dn1, _ = A1.shape
        dn2 = A2.shape[2]
        _, _, dn3, dr = A3.shape
        rk = len(kraus)
        K = np.stack([N @ U for N in kraus]).reshape(rk, 2, 2, 2, 2, 2, 2)  # [k, a', b', c', a, b, c]
        th = np.einsum("lanx,xbmy,ycor->lanbmcor", A1, A2, A3)            # [l, p1, n1, p2, n2, p3, n3, r]
        th = np.einsum("kxyzabc,lanbmcor->lxnymzkor", K, th)              # [l, p1', n1, p2', n2, p3', k, n3, r]
        dk = rk * dn3
        mat = self._perturbed(th.reshape(dl * 2 * dn1, -1))
        Um, s, Vh = np.linalg.svd(mat, full_matrices=False)
        k1, w1 = self._keep(s, self.chi_max)
        self.sites[q] = Um[:, :k1].reshape(dl, 2, dn1, k1)
        self.discarded_chi += w1
        self.log.append(("chi", q, k1, len(s), w1))
        rest = self._perturbed((s[:k1, None] * Vh[:k1]).reshape(k1 * 2 * dn2, 2 * dk * dr))
        Um2, s2, Vh2 = np.linalg.svd(rest, full_matrices=False)
        k2, w2 = self._keep(s2, self.chi_max)
        self.sites[q + 1] = Um2[:, :k2].reshape(k1, 2, dn2, k2)
        self.sites[q + 2] = (s2[:k2, None] * Vh2[:k2]).reshape(k2, 2, dk, dr)
        self.discarded_chi += w2
        self.log.append(("chi", q + 1, k2, len(s2), w2))
        self.centre = q + 2
        if self.auto_truncate:
            self.truncate_kraus(q + 2)

    # ------------------------------------------------------------ readouts
    def _bra_ket(self, ops) -> complex:
        """sum_n <psi_n| (x)_i O_i |psi_n>, O_i = ops.get(i, I); E'[r,r'] = sum E[l,l'] T*[l,p,n,r] O[p,p'] T[l',p',n,r']."""
        E = np.ones((1, 1), dtype=np.complex128)
        for i, A in enumerate(self.sites):
            O = ops.get(i)
            B = A if O is None else np.einsum("ab,lbnr->lanr", O, A)
            X = np.einsum("xy,xpnr->ypnr", E, A.conj(), optimize=True)
            E = np.einsum("ypnr,ypns->rs", X, B, optimize=True)
        return complex(E[0, 0])

    def trace(self) -> float:
        return self._bra_ket({}).real

    def expect_product(self, ops) -> float:
        return self._bra_ket(ops).real / self.trace()

    def expect_zz(self, i: int, j: int) -> float:
        Z = np.diag([1.0, -1.0]).astype(np.complex128)
        return self.expect_product({i: Z, j: Z})

    def zz_map(self) -> np.ndarray:
        out = np.zeros((self.n, self.n))
        for i in range(self.n):
            out[i, i] = 1.0
            for j in range(i + 1, self.n):
                out[i, j] = out[j, i] = self.expect_zz(i, j)
        return out

    def element(self, a, b) -> complex:
        """<a| rho |b> for computational basis strings a, b: E'[r,r'] = sum E[l,l'] T[l,a_i,n,r] T*[l',b_i,n,r']."""
        E = np.ones((1, 1), dtype=np.complex128)
        for i, A in enumerate(self.sites):
            X = np.einsum("xy,xnr->ynr", E, A[:, a[i]], optimize=True)
            E = np.einsum("ynr,yns->rs", X, A[:, b[i]].conj(), optimize=True)
        return complex(E[0, 0])

    def ghz_fidelity(self) -> float:
        z, o = [0] * self.n, [1] * self.n
        f = 0.5 * (self.element(z, z) + self.element(o, o) + 2 * self.element(z, o)).real
        return f / self.trace()

    def maxcut(self, edges) -> float:
        return sum(0.5 * (1 - self.expect_zz(i, k)) for i, k in edges)

    def purity(self) -> float:
        """Tr(rho^2) / Tr(rho)^2 with rho_pq rho_qp contracted through a four-copy transfer."""
        E = np.ones((1, 1, 1, 1), dtype=np.complex128)
        for A in self.sites:
            Ac = A.conj()
            # one copy at a time (pairwise contractions, each a single BLAS product)
            X = np.einsum("abcd,apnr->bcdpnr", E, A, optimize=True)        # copy 1, ket
            X = np.einsum("bcdpnr,bqns->cdprqs", X, Ac, optimize=True)     # copy 1, bra (Kraus leg n summed)
            X = np.einsum("cdprqs,cqmt->dprsmt", X, A, optimize=True)      # copy 2, ket
            E = np.einsum("dprsmt,dpmu->rstu", X, Ac, optimize=True)       # copy 2, bra (Kraus leg m summed)
        return E[0, 0, 0, 0].real / self.trace() ** 2

    def dense(self) -> np.ndarray:
        """rho = sum_n |psi_n><psi_n| as a 2^n x 2^n matrix (small n only), accumulated site by site
        as R[P, P', r, r'] = sum R[P, P', l, l'] T[l, p, n, r] T*[l', p', n, r'] (Kraus legs summed)."""
        R = np.ones((1, 1, 1, 1), dtype=np.complex128)
        for A in self.sites:
            R = np.einsum("abxy,xpnr->abypnr", R, A)
            R = np.einsum("abypnr,yqns->apbqrs", R, A.conj())
            s = R.shape
            R = R.reshape(s[0] * 2, s[2] * 2, s[4], s[5])
        return R[:, :, 0, 0]

    def bond_dims(self):
        return [A.shape[3] for A in self.sites[:-1]]

    def kraus_dims(self):
        return [A.shape[2] for A in self.sites]


def run_circuit(circuit, chi_max: int, kappa_max: int, tol: float = 1e-13, kraus_tol: float = 1e-12,
                perturb=None, trunc_order: str = "split_first") -> MPDO:
    """Convert every channel from its chi matrix (Sec. III) and apply the ops in order."""
    kraus = [chi_to_kraus(chi, nq, kraus_tol) for nq, chi in circuit.chis]
    st = MPDO(circuit.n, chi_max, kappa_max, tol, trunc_order=trunc_order)
    st.perturb = perturb
    for op in circuit.ops:
        if op.kind == 8:
            st.truncate_bonds(op.q)
        elif op.kind == 1:
            st.apply_1q(op.q, op.U, kraus[op.chan])
        elif op.kind == 3:
            st.apply_3q(op.q, op.U, kraus[op.chan])
        else:
            st.apply_2q(op.q, op.U, kraus[op.chan])
    return st
