"""Sequential HIF-IE in 2D and 3D (oracle; test infrastructure).

Follows the paper's steps in its own order and notation:

* Algorithm 4.1 (2D: cells at level l, edges at l + 1/2) and Algorithm 4.2
  (3D: cells, faces at l + 1/3, edges at l + 2/3); with ``fractional=False``
  it is RSF, Algorithm 3.1.
* Skeletonization of one index set c (Lemma 2.4): ID of the proxy matrix Y_c
  (Eq. (3.3): near-field rows A_{cN,c}, A_{c,cN}^T and proxy rows Y_{cE,c},
  Y_{c,cE}^T, Sec. 3.3 Lemma 3.3 with quadrature weights), then elimination
  of the redundant DOFs by Lemma 2.1 with the B blocks of Lemma 2.4.
* Near field (Sec. 3.3 and 4.3): active DOFs strictly inside the proxy
  circle/sphere of radius 1.5 w about the box centre, plus every active DOF
  coupled to c through a Schur-complement interaction (SCI).
* Second-kind modifications (Sec. 4.4): columns grouped by the structural
  sparsity pattern of Y^S_c (Lemma 4.2), each group compressed on its own
  with tolerance rho_g eps, rho_g = min(1, |Y^K_g| / |Y^S_g|).
* The factorization F of Eqs. (4.1)/(4.2) is applied in factored form:
  ``apply`` = F x, ``solve`` = F^{-1} x and their transposes (Sec. 3.1: each
  unit-triangular factor is inverted by negating its off-diagonal block).

The active matrix A_l is held as the dense sum A + S, where S accumulates the
Schur updates and the boolean matrix M records their structure, so that every
block the paper names is read straight out of a dense array.  This limits the
oracle to a few thousand DOFs, which is what it is for.

Readings of points the paper leaves open (the GPU path uses the same ones):
 1. Root box: the bounding cube of the DOFs' cells (side w_j^(1/d) about x_j);
    L = the smallest depth at which no cell holds more than ``occupancy`` DOFs.
    Level l uses s = 2^(L-l) cells per side of width w = W / s.
 2. Cells: DOF -> cell floor((x - lo) / w), clamped to [0, s-1] (a point on a
    split plane goes to the upper cell).  Edges/faces: only interior ones
    exist (Sec. 4.1/4.2 index ranges); each active DOF joins the nearest
    centre by squared distance; centres within a relative TIE = 2^-40 of the
    smallest squared distance count as tied, and the lowest centre id wins
    (on a grid, tied centres are exactly equidistant, but their computed
    distances can differ by rounding: three squares summed in different
    orders, or a cube root for the root box's cell side that is not
    correctly rounded everywhere).  Centre ids:
    the paper's listing order of the families (2D edges: x-normal then
    y-normal; 3D faces: x-, y-, z-normal; 3D edges: z-, y-, x-directed),
    lexicographic with the first index slowest inside each family.
 3. Processing inside one sublevel is level-synchronous: the near field of
    every box is taken from the active set at the start of the sublevel.
 4. Y_c row order: [A_{cN,c}; A_{c,cN}^T; proxy-out; proxy-in].  Proxy-out
    entries G(|x^E_k - x_j|) w_j c_j, proxy-in entries b_j G(|x_j - x^E_k|) w_j.
 5. Groups: columns with identical structural SCI pattern over the near-field
    rows (a column with no SCI forms part of the empty-pattern group); group
    order = first appearance in ascending DOF order.  With second_kind off
    there is one group and rho = 1.  rho_g = 1 when the group has no SCI.
 6. Column order inside a box: ascending global DOF id.  Skeletons: groups in
    order, each in pivot order; redundants: groups in order, each ascending.
 7. A Schur update is recorded (S and M over skel x skel) only when the box
    eliminated something and kept a skeleton.
 8. Symmetry (Sec. 5, opening paragraph): when A is symmetric the one-sided
    Y'_c = [A_{cN,c}; Y_{cE,c}] is compressed instead of Y_c.  A is taken
    as symmetric when b = c entrywise and all weights w_j are equal, the
    sufficient form of b_i w_j c_j = b_j w_i c_i for all i != j.  The
    dropped rows repeat the kept ones (the active matrix A + S stays
    symmetric under symmetric elimination), so Y_c^T Y_c = 2 Y'_c^T Y'_c and
    the pivoted QR picks the same skeletons with the same T.
 9. LDL (Sec. 5, opening paragraph: symmetric diagonal blocks are factored
    by a partially pivoted LDL).  For symmetric A, B_rr is factored as
    P B_rr P^T = L D L^T with 1 x 1 symmetric pivots: at each step the
    remaining diagonal entry of largest magnitude (ties: lowest position),
    accepted when it is at least alpha = (1 + sqrt 17) / 8 times the largest
    other entry of its column (the Bunch-Kaufman test for a 1 x 1 pivot).
    A box whose pivot fails the test is factored by LU with partial pivoting
    instead (2 x 2 pivots are not used).  With U = L^T P the factored form
    is the LU one, P B_rr = L D U, and Y = D^{-1} L^{-1} P B_rs = X^T, so
    only X is kept; the Schur update -X D X^T is symmetric by construction.
10. Helmholtz (Sec. 5, Example 3): complex arithmetic is carried out in the
    real 2 x 2 embedding z -> [[Re z, -Im z], [Im z, Re z]] (oracle/helmholtz.py):
    DOF j becomes real DOFs 2j, 2j + 1 at the same point, the proxy surface
    contributes two rows per point and direction, and the whole method runs
    unchanged on the real operator.  Its transposes are the complex adjoints.
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np
from scipy.linalg import lu as dense_lu, lu_factor, lu_solve, solve_triangular

from .idqr import interp_decomp, norm2_estimate
from .kernels import Operator, green

_H, _I = "h", "i"
TIE = 2.0 ** -40          # relative squared-distance difference counted as a tie (reading 2)
FAMILIES = {
    (2, "cell"): [(_H, _H)],
    (2, "edge"): [(_I, _H), (_H, _I)],
    (3, "cell"): [(_H, _H, _H)],
    (3, "face"): [(_I, _H, _H), (_H, _I, _H), (_H, _H, _I)],
    (3, "edge"): [(_I, _I, _H), (_I, _H, _I), (_H, _I, _I)],
}


def root_box(points: np.ndarray, weights: np.ndarray):
    d = points.shape[1]
    side = np.sqrt(weights) if d == 2 else np.cbrt(weights)
    lo = (points - 0.5 * side[:, None]).min(axis=0)
    hi = (points + 0.5 * side[:, None]).max(axis=0)
    return lo, float((hi - lo).max())


def cell_index(points, lo, W, s):
    w = W / s
    t = np.floor((points - lo[None, :]) / w).astype(np.int64)
    return np.clip(t, 0, s - 1)


def num_levels(points, lo, W, occupancy: int, max_levels: int = 24) -> int:
    d = points.shape[1]
    for L in range(max_levels + 1):
        s = 2**L
        t = cell_index(points, lo, W, s)
        flat = np.zeros(len(points), dtype=np.int64)
        for k in range(d):
            flat = flat * s + t[:, k]
        if np.bincount(flat).max() <= occupancy:
            return L
    return max_levels


def centers(kind: str, d: int, s: int, lo: np.ndarray, w: float) -> np.ndarray:
    out = []
    for fam in FAMILIES[(d, kind)]:
        ranges = [range(1, s) if t == _I else range(0, s) for t in fam]
        for js in itertools.product(*ranges):
            out.append([lo[k] + (js[k] + (0.5 if fam[k] == _H else 0.0)) * w for k in range(d)])
    return np.asarray(out, dtype=np.float64).reshape(-1, d)


@dataclass
class BoxFactor:
    sk: np.ndarray      # skeleton DOFs (global ids)
    rd: np.ndarray      # redundant DOFs (global ids)
    T: np.ndarray       # k x r interpolation matrix (block diagonal over groups)
    L: np.ndarray       # r x r unit lower triangular
    D: np.ndarray       # r diagonal
    U: np.ndarray       # r x r unit upper triangular
    perm: np.ndarray    # P B_rr = L D U with (P x)_i = x[perm[i]]
    X: np.ndarray       # k x r : B_sr U^{-1} D^{-1}
    Y: np.ndarray       # r x k : D^{-1} L^{-1} P B_rs
    ngroups: int = 1
    n: int = 0
    m: int = 0
    ldl: bool = False   # P B_rr P^T = L D L^T: U = L^T P (dense, not triangular), Y = X^T

    def U_solve(self, v, trans=False):
        """U^{-1} v (U^{-T} v with trans) for either factor form."""
        if not self.ldl:
            return solve_triangular(self.U, v, lower=False, trans=1 if trans else 0, unit_diagonal=True)
        if trans:                                    # U^{-T} = L^{-1} P
            return solve_triangular(self.L, v[self.perm], lower=True, unit_diagonal=True)
        w = solve_triangular(self.L, v, lower=True, trans=1, unit_diagonal=True)   # U^{-1} = P^T L^{-T}
        out = np.empty_like(w)
        out[self.perm] = w
        return out


@dataclass
class Sublevel:
    kind: str
    level: int
    boxes: list = field(default_factory=list)


@dataclass
class HIFFactor:
    N: int
    sublevels: list
    top: np.ndarray          # s_L, global ids ascending
    top_A: np.ndarray        # A_L restricted to s_L
    top_lu: tuple

    # ---- statistics (Sec. 5 column definitions) ----
    @property
    def sL(self) -> int:
        return int(self.top.size)

    def storage_doubles(self) -> int:
        tot = self.top.size ** 2
        for sl in self.sublevels:
            for bf in sl.boxes:
                k, r = bf.sk.size, bf.rd.size
                # LU: T, X, Y, L and U, D; LDL: T, X, strict L, D
                tot += (2 * k * r + r * (r - 1) // 2 + r) if bf.ldl else (3 * k * r + r * r + r)
        return int(tot)

    def ranks(self):
        return [(sl.kind, sl.level, len(sl.boxes), sum(b.sk.size for b in sl.boxes),
                 sum(b.rd.size for b in sl.boxes)) for sl in self.sublevels]

    # ---- factored-form application (Eqs. (3.2), (4.1), (4.2)) ----
    def _boxes(self, reverse=False):
        sls = reversed(self.sublevels) if reverse else self.sublevels
        for sl in sls:
            for bf in sl.boxes:
                if bf.rd.size:
                    yield bf

    def solve(self, b):
        """x = F^{-1} b = V_0 ... V_last D^{-1} U_last^T ... U_0^T b."""
        x = np.array(b, dtype=np.float64, copy=True)
        for bf in self._boxes():                         # U^T, finest first
            x[bf.rd] -= bf.T.T @ x[bf.sk]
            x[bf.rd] = solve_triangular(bf.L, x[bf.rd][bf.perm], lower=True, unit_diagonal=True)
            x[bf.sk] -= bf.X @ x[bf.rd]
        for bf in self._boxes():                         # D^{-1}
            x[bf.rd] = (x[bf.rd].T / bf.D).T
        if self.top.size:
            x[self.top] = lu_solve(self.top_lu, x[self.top])
        for bf in self._boxes(reverse=True):             # V, coarsest first
            x[bf.rd] -= bf.Y @ x[bf.sk]
            x[bf.rd] = bf.U_solve(x[bf.rd])
            x[bf.sk] -= bf.T @ x[bf.rd]
        return x

    def apply(self, v):
        """y = F v = U_0^{-T} ... U_last^{-T} D V_last^{-1} ... V_0^{-1} v."""
        x = np.array(v, dtype=np.float64, copy=True)
        for bf in self._boxes():                         # V^{-1}, finest first
            x[bf.sk] += bf.T @ x[bf.rd]
            x[bf.rd] = bf.U @ x[bf.rd]
            x[bf.rd] += bf.Y @ x[bf.sk]
        for bf in self._boxes():                         # D
            x[bf.rd] = (x[bf.rd].T * bf.D).T
        if self.top.size:
            x[self.top] = self.top_A @ x[self.top]
        for bf in self._boxes(reverse=True):             # U^{-T}, coarsest first
            x[bf.sk] += bf.X @ x[bf.rd]
            y = bf.L @ x[bf.rd]
            tmp = np.empty_like(y)
            tmp[bf.perm] = y                             # P^T
            x[bf.rd] = tmp
            x[bf.rd] += bf.T.T @ x[bf.sk]
        return x

    def solve_transpose(self, b):
        """x = F^{-T} b = U_0 ... U_last D^{-T} V_last^T ... V_0^T b."""
        x = np.array(b, dtype=np.float64, copy=True)
        for bf in self._boxes():                         # V^T, finest first
            x[bf.rd] -= bf.T.T @ x[bf.sk]
            x[bf.rd] = bf.U_solve(x[bf.rd], trans=True)
            x[bf.sk] -= bf.Y.T @ x[bf.rd]
        for bf in self._boxes():                         # D^{-T}
            x[bf.rd] = (x[bf.rd].T / bf.D).T
        if self.top.size:
            x[self.top] = lu_solve(self.top_lu, x[self.top], trans=1)
        for bf in self._boxes(reverse=True):             # U, coarsest first
            x[bf.rd] -= bf.X.T @ x[bf.sk]
            y = solve_triangular(bf.L, x[bf.rd], lower=True, trans=1, unit_diagonal=True)
            tmp = np.empty_like(y)
            tmp[bf.perm] = y                             # P^T
            x[bf.rd] = tmp
            x[bf.sk] -= bf.T @ x[bf.rd]
        return x

    def apply_transpose(self, v):
        """y = F^T v = V_0^{-T} ... V_last^{-T} D^T U_last^{-1} ... U_0^{-1} v."""
        x = np.array(v, dtype=np.float64, copy=True)
        for bf in self._boxes():                         # U^{-1}, finest first
            x[bf.sk] += bf.T @ x[bf.rd]
            x[bf.rd] = bf.L.T @ x[bf.rd][bf.perm]
            x[bf.rd] += bf.X.T @ x[bf.sk]
        for bf in self._boxes():                         # D^T
            x[bf.rd] = (x[bf.rd].T * bf.D).T
        if self.top.size:
            x[self.top] = self.top_A.T @ x[self.top]
        for bf in self._boxes(reverse=True):             # V^{-T}, coarsest first
            x[bf.sk] += bf.Y.T @ x[bf.rd]
            x[bf.rd] = bf.U.T @ x[bf.rd]
            x[bf.rd] += bf.T.T @ x[bf.sk]
        return x

    # ---- explicit products, for checking the sweeps on tiny problems ----
    def dense_factors(self):
        """Dense N x N matrices (U_tau, V_tau per sublevel, D) of Eq. (4.1)."""
        N = self.N
        Us, Vs = [], []
        D = np.zeros((N, N))
        for sl in self.sublevels:
            Ut = np.eye(N)
            Vt = np.eye(N)
            for bf in sl.boxes:
                if not bf.rd.size:
                    continue
                rd, sk = bf.rd, bf.sk
                Q = np.eye(N)
                Q[np.ix_(sk, rd)] = -bf.T
                Lp = np.zeros((rd.size, rd.size))
                Lp[bf.perm, :] = bf.L                    # L_p = P^T L
                Rs = np.eye(N)                           # R^* = [I;-X I] diag(L_p^{-1})
                Rs[np.ix_(rd, rd)] = np.linalg.inv(Lp)
                E = np.eye(N)
                E[np.ix_(sk, rd)] = -bf.X
                Rs = E @ Rs
                S = np.eye(N)                            # S = diag(U^{-1}) [I -Y; I]
                S[np.ix_(rd, rd)] = np.linalg.inv(bf.U)
                E2 = np.eye(N)
                E2[np.ix_(rd, sk)] = -bf.Y
                S = S @ E2
                Ut = Ut @ (Q @ Rs.T)
                Vt = Vt @ (Q @ S)
                D[np.ix_(rd, rd)] = np.diag(bf.D)
            Us.append(Ut)
            Vs.append(Vt)
        if self.top.size:
            D[np.ix_(self.top, self.top)] = self.top_A
        return Us, Vs, D

    def dense_F(self):
        Us, Vs, D = self.dense_factors()
        F = D
        for Ut, Vt in zip(reversed(Us), reversed(Vs)):
            F = np.linalg.inv(Ut).T @ F @ np.linalg.inv(Vt)
        return F


def sublevel_plan(dim: int, L: int, fractional: bool = True, skip_levels: int = 0):
    plan = []
    for ell in range(L):
        plan.append(("cell", ell))
        if fractional and ell >= skip_levels:
            if dim == 2:
                plan.append(("edge", ell))
            else:
                plan.append(("face", ell))
                plan.append(("edge", ell))
    return plan


def factor(points, weights, a, b, c, kernel_id: int, eps: float, proxy_dirs,
           *, second_kind: bool = True, occupancy: int = 64, proxy_radius: float = 1.5,
           fractional: bool = True, skip_levels: int = 0, symmetric=None, ldl=None,
           wavenumber=None, trace=None, trace_sets=None) -> HIFFactor:
    """HIF-IE (Algorithm 4.1 / 4.2) of A = diag(a) + diag(b) K diag(c).

    ``symmetric``: None compresses Y'_c exactly when ``is_symmetric`` holds,
    False always compresses the full Y_c, True requires ``is_symmetric``.
    ``ldl``: None factors B_rr by LDL exactly when Y'_c is compressed
    (reading 9), False always by LU.
    kernel_id 2 (Helmholtz, Sec. 5 Example 3, wavenumber k): the factorization
    runs on the real 2 x 2 embedding of the complex operator (reading 10), on
    2N real DOFs, two at every point; occupancy counts real DOFs.
    ``trace_sets`` (a list) receives, box by box, the index sets of every
    skeletonization: (kind, level, box DOFs c, near field c^N, column groups,
    skeletons, redundants), all global ids.
    """
    if kernel_id == 2:
        from .helmholtz import EmbeddedOperator
        op = EmbeddedOperator(points, weights, a, b, c, wavenumber)
    else:
        op = Operator(points, weights, a, b, c, kernel_id)
    if symmetric is None:
        symmetric = is_symmetric(op)
    elif symmetric and not is_symmetric(op):
        raise ValueError("symmetric=True needs b == c and equal weights")
    use_ldl = bool(symmetric) if ldl is None else (bool(ldl) and bool(symmetric))
    x = op.x
    N, d = x.shape
    proxy_dirs = np.asarray(proxy_dirs, dtype=np.float64)
    P = proxy_dirs.shape[0]
    lo, W = root_box(x, op.w)
    L = num_levels(x, lo, W, occupancy)

    S = np.zeros((N, N))                 # accumulated Schur-complement interactions
    M = np.zeros((N, N), dtype=bool)     # their structure
    active = np.ones(N, dtype=bool)
    sublevels = []

    for kind, ell in sublevel_plan(d, L, fractional, skip_levels):
        s = 2 ** (L - ell)
        w = W / s
        act_idx = np.nonzero(active)[0]
        if kind == "cell":
            t = cell_index(x[act_idx], lo, W, s)
            flat = np.zeros(act_idx.size, dtype=np.int64)
            for k in range(d):
                flat = flat * s + t[:, k]
            ctr = centers("cell", d, s, lo, w)
            owner = flat
        else:
            ctr = centers(kind, d, s, lo, w)
            diff = x[act_idx][:, None, :] - ctr[None, :, :]
            dist2 = (diff * diff).sum(axis=2)
            best = dist2.min(axis=1, keepdims=True)
            owner = np.argmax(dist2 <= best * (1.0 + TIE), axis=1)    # first tied centre = lowest id
        snapshot = active.copy()                       # level-synchronous reading
        R2 = (proxy_radius * w) ** 2
        sl = Sublevel(kind=kind, level=ell)
        for bid in range(ctr.shape[0]):
            cbox = act_idx[owner == bid]
            if cbox.size == 0:
                continue
            sets = {} if trace_sets is not None else None
            bf = _skeletonize(op, S, M, snapshot, cbox, ctr[bid], R2, proxy_radius * w,
                              proxy_dirs, eps, second_kind, bool(symmetric), use_ldl, sets)
            sl.boxes.append(bf)
            active[bf.rd] = False
            if trace is not None:
                trace.append((kind, ell, bid, cbox.size, bf.sk.size, bf.m, bf.ngroups))
            if trace_sets is not None:
                trace_sets.append((kind, ell, cbox, sets["near"], sets["groups"], bf.sk, bf.rd))
        sublevels.append(sl)

    top = np.nonzero(active)[0]
    top_A = op.entries(top, top) + S[np.ix_(top, top)]
    top_lu = lu_factor(top_A) if top.size else None
    return HIFFactor(N=N, sublevels=sublevels, top=top, top_A=top_A, top_lu=top_lu)


def is_symmetric(op: Operator) -> bool:
    """Sufficient test for A = A^T: b = c entrywise and equal weights.  The
    real embedding of a complex symmetric matrix is not symmetric (its
    transpose embeds the conjugate transpose)."""
    if op.kernel_id == 2:
        return False
    return bool(np.array_equal(op.b, op.c) and np.all(op.w == op.w[0]))


def sci_groups(pattern: np.ndarray):
    """Split the columns of a boolean pattern matrix into groups of identical
    columns (Sec. 4.4); groups ordered by first appearance."""
    keys = {}
    gid = np.empty(pattern.shape[1], dtype=np.int64)
    for j in range(pattern.shape[1]):
        key = pattern[:, j].tobytes()
        if key not in keys:
            keys[key] = len(keys)
        gid[j] = keys[key]
    return [np.nonzero(gid == g)[0] for g in range(len(keys))]


LDL_ALPHA = (1.0 + np.sqrt(17.0)) / 8.0


def ldl_diag_pivot(B):
    """P B P^T = L D L^T with 1 x 1 symmetric pivots (reading 9).

    Returns (perm, L, D) with (P x)_i = x[perm[i]], or None when a pivot
    fails the test |B_pp| >= alpha * max_{i != p} |B_ip| (or is zero)."""
    Bw = np.array(B, dtype=np.float64, copy=True)
    r = Bw.shape[0]
    perm = np.arange(r)
    L = np.eye(r)
    D = np.zeros(r)
    for j in range(r):
        diag = np.abs(np.diag(Bw)[j:])
        p = j + int(np.argmax(diag))                 # first maximum = lowest position
        col = np.abs(Bw[j:, p])
        col[p - j] = 0.0
        colmax = col.max() if col.size else 0.0
        if Bw[p, p] == 0.0 or not np.isfinite(Bw[p, p]) or abs(Bw[p, p]) < LDL_ALPHA * colmax:
            return None
        if p != j:                                   # symmetric interchange of rows and columns j, p
            Bw[[j, p], :] = Bw[[p, j], :]
            Bw[:, [j, p]] = Bw[:, [p, j]]
            L[[j, p], :j] = L[[p, j], :j]
            perm[[j, p]] = perm[[p, j]]
        D[j] = Bw[j, j]
        L[j + 1:, j] = Bw[j + 1:, j] / D[j]
        Bw[j + 1:, j + 1:] -= D[j] * np.outer(L[j + 1:, j], L[j + 1:, j])
    return perm, L, D


def _skeletonize(op: Operator, S, M, snapshot, cbox, center, R2, radius, proxy_dirs,
                 eps, second_kind, symmetric=False, use_ldl=False, sets=None) -> BoxFactor:
    x = op.x
    n = cbox.size
    inbox = np.zeros(op.N, dtype=bool)
    inbox[cbox] = True
    cand = snapshot & ~inbox
    diff = x - center[None, :]
    # strictly inside: within a relative TIE of the radius counts as on it
    # (grids put DOFs exactly on the proxy sphere; rounding must not decide)
    near = cand & ((diff * diff).sum(axis=1) < R2 * (1.0 - TIE))
    sci = cand & M[:, cbox].any(axis=1)
    cN = np.nonzero(near | sci)[0]

    # Y_c of Eq. (3.3), split as Y^K (kernel + proxy) and Y^S (SCI); for a
    # symmetric A the one-sided Y'_c of Sec. 5 (reading 8)
    xE = center[None, :] + radius * proxy_dirs
    YK_near1 = op.kernel_entries(cN, cbox)
    YK_out = op.proxy_out(xE, cbox)
    if symmetric:
        YK = np.vstack([YK_near1, YK_out])
        YS = np.vstack([S[np.ix_(cN, cbox)], np.zeros((YK_out.shape[0], n))])
    else:
        YK_near2 = op.kernel_entries(cbox, cN).T
        YK_in = op.proxy_in(xE, cbox)
        YK = np.vstack([YK_near1, YK_near2, YK_out, YK_in])
        YS = np.vstack([S[np.ix_(cN, cbox)], S[np.ix_(cbox, cN)].T,
                        np.zeros((YK_out.shape[0] + YK_in.shape[0], n))])
    Y = YK + YS
    m = Y.shape[0]

    # groups by structural SCI pattern (Lemma 4.2)
    groups = sci_groups(M[np.ix_(cN, cbox)]) if second_kind else [np.arange(n)]
    if sets is not None:
        sets["near"] = cN.copy()
        sets["groups"] = [cbox[g] for g in groups]

    sk_l, rd_l, T_blocks = [], [], []
    for g in groups:
        rho = 1.0
        if second_kind and M[np.ix_(cN, cbox[g])].any():
            nS = norm2_estimate(YS[:, g])
            nK = norm2_estimate(YK[:, g])
            if nS > 0.0:
                rho = min(1.0, nK / nS)
        sk, rd, T = interp_decomp(Y[:, g], rho * eps)
        sk_l.append(g[sk])
        rd_l.append(g[rd])
        T_blocks.append(T)
    sk_loc = np.concatenate(sk_l) if sk_l else np.zeros(0, dtype=np.int64)
    rd_loc = np.concatenate(rd_l) if rd_l else np.zeros(0, dtype=np.int64)
    k, r = sk_loc.size, rd_loc.size
    T = np.zeros((k, r))
    ko = ro = 0
    for Tg in T_blocks:
        T[ko:ko + Tg.shape[0], ro:ro + Tg.shape[1]] = Tg
        ko += Tg.shape[0]
        ro += Tg.shape[1]
    sk_g, rd_g = cbox[sk_loc], cbox[rd_loc]

    if r == 0:
        z = np.zeros((0, 0))
        return BoxFactor(sk=sk_g, rd=rd_g, T=T, L=z, D=np.zeros(0), U=z,
                         perm=np.zeros(0, dtype=np.int64), X=np.zeros((k, 0)),
                         Y=np.zeros((0, k)), ngroups=len(groups), n=n, m=m)

    def Ablk(I, J):
        return op.entries(I, J) + S[np.ix_(I, J)]

    A_rr, A_rs = Ablk(rd_g, rd_g), Ablk(rd_g, sk_g)
    A_sr, A_ss = Ablk(sk_g, rd_g), Ablk(sk_g, sk_g)
    # Lemma 2.4 blocks (real case: * = transpose)
    B_rr = A_rr - T.T @ A_sr - A_rs @ T + T.T @ A_ss @ T
    B_rs = A_rs - T.T @ A_ss
    B_sr = A_sr - A_ss @ T
    fac = ldl_diag_pivot(B_rr) if use_ldl else None
    if fac is not None:
        # reading 9: P B_rr P^T = L D L^T, U = L^T P, X = B_sr P^T L^{-T} D^{-1}, Y = X^T
        perm, Lm, Dg = fac
        inv = np.empty_like(perm)
        inv[perm] = np.arange(perm.size)
        Um = Lm.T[:, inv]
        Xp = solve_triangular(Lm, B_sr[:, perm].T, lower=True, unit_diagonal=True).T
        X = Xp / Dg[None, :]
        if k > 0:
            delta = -(X * Dg[None, :]) @ X.T
            S[np.ix_(sk_g, sk_g)] += delta
            M[np.ix_(sk_g, sk_g)] = True
        return BoxFactor(sk=sk_g, rd=rd_g, T=T, L=Lm, D=Dg, U=Um, perm=perm, X=X, Y=X.T.copy(),
                         ngroups=len(groups), n=n, m=m, ldl=True)
    # Lemma 2.1 on B_rr with partial pivoting: P B_rr = L D U
    Pm, Lm, Ut = dense_lu(B_rr)
    perm = Pm.argmax(axis=0)
    Dg = np.diag(Ut).copy()
    if np.any(Dg == 0.0) or not np.all(np.isfinite(Dg)):
        raise np.linalg.LinAlgError("singular B_rr in skeletonization")
    Um = Ut / Dg[:, None]
    X = solve_triangular(Ut, B_sr.T, trans=1, lower=False).T
    Yf = solve_triangular(Lm, B_rs[perm], lower=True, unit_diagonal=True) / Dg[:, None]
    if k > 0:
        delta = -B_sr @ np.linalg.solve(B_rr, B_rs)
        S[np.ix_(sk_g, sk_g)] += delta
        M[np.ix_(sk_g, sk_g)] = True
    return BoxFactor(sk=sk_g, rd=rd_g, T=T, L=Lm, D=Dg, U=Um, perm=perm, X=X, Y=Yf,
                     ngroups=len(groups), n=n, m=m)
