"""Plain numpy / Python oracle for ALTO (test infrastructure only).

Everything here is fp64 (or exact integers) and follows the paper's text in
the order it states the steps. Only tests/, __graft_entry__.smoke() and
bench.py's CPU legs may use it.

Readings of the paper that this file fixes:

* Coordinates are 0-based, as in the worked example of Fig. 3(a).
* "log2 I_n" bits per mode (Eq. 1) is bit_width(I_n - 1): the smallest b with
  2^b >= I_n, so a mode of length 1 takes no bits.
* Bit groups fill the linear index from the least significant bit; group g
  holds bit g of every mode that still has bits left; inside a group the
  modes come in increasing order of their length I_n (ties: lower mode index
  first), the shortest at the lowest bit (Section III-A, "shortest mode
  first"). The printed line segments [2-20] / [25-51] of Section IV-A only
  come out with this order.
* The ordering step is a stable sort by the linear index; equal indices keep
  their input order.
* Line segment l of L holds positions [floor(l*M/L), floor((l+1)*M/L)) of the
  ordered tensor ("the same number of nonzero elements", Section IV-A). An
  empty segment gets the empty interval (2^32-1, 0) in every mode.
* CP-ALS (Alg. 1): the pseudo-inverse is taken through a Cholesky solve when V
  is positive definite, else numpy's pinv; "column normalize" uses 2-norms
  every iteration, a zero column (norm at most 1e-12 of the largest column's,
  i.e. rounding noise of a pseudo-inverse solve) gets lambda 0 and is set to
  zero; the fit is
  1 - ||X - X_hat|| / ||X|| evaluated with the usual expansion
  ||X||^2 + lambda^T (*_m G_m) lambda - 2 <X, X_hat>.
* Duplicate coordinates are separate COO entries that add up into one cell of
  X: MTTKRP sums them term by term, and ||X||^2 squares the summed cells.
* pos_out of Alg. 4 (the output-oriented traversal) lists, segment by
  segment, the ordered positions of the segment by increasing coordinate of
  the output mode; equal coordinates keep line order. Segments are those of
  Section IV-A for a given L. A row is a boundary row of a segment when
  another segment also has nonzeros in it: only those updates need atomics.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

EMPTY_LO = 0xFFFFFFFF


# ---------------------------------------------------------------------------
# Section III-A: bit plan, linearization (bit gather), de-linearization
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class BitPlan:
    dims: Tuple[int, ...]
    bits: Tuple[int, ...]                 # bits per mode
    order: Tuple[int, ...]                # modes, shortest first
    positions: Tuple[Tuple[int, ...], ...]  # positions[n][g] = key bit of bit g of mode n
    nbits: int
    masks: Tuple[int, ...]                # one mask per mode (Python int)

    @property
    def nmodes(self) -> int:
        return len(self.dims)


def mode_bits(I: int) -> int:
    """Bits needed for coordinates 0..I-1 (0 for a mode of length 1)."""
    if I < 1:
        raise ValueError("mode length must be >= 1")
    return int(I - 1).bit_length()


def bit_plan(dims: Sequence[int]) -> BitPlan:
    """Section III-A: group bits from the LSB, shortest mode first per group."""
    dims = tuple(int(d) for d in dims)
    bits = tuple(mode_bits(I) for I in dims)
    order = tuple(sorted(range(len(dims)), key=lambda n: (dims[n], n)))
    positions: List[List[int]] = [[] for _ in dims]
    p = 0
    for g in range(max(bits) if bits else 0):
        for n in order:
            if bits[n] > g:
                positions[n].append(p)
                p += 1
    masks = tuple(sum(1 << q for q in positions[n]) for n in range(len(dims)))
    return BitPlan(dims, bits, order, tuple(tuple(x) for x in positions), p, masks)


def linearize_one(index: Sequence[int], plan: BitPlan) -> int:
    """Bit-level gather of one coordinate tuple into its line position."""
    key = 0
    for n, i in enumerate(index):
        for g, q in enumerate(plan.positions[n]):
            key |= ((int(i) >> g) & 1) << q
    return key


def delinearize_one(key: int, plan: BitPlan) -> Tuple[int, ...]:
    """Bit-level scatter: EXTRACT(p, MASK) of Alg. 3, one mode at a time."""
    out = []
    for n in range(plan.nmodes):
        i = 0
        for g, q in enumerate(plan.positions[n]):
            i |= ((key >> q) & 1) << g
        out.append(i)
    return tuple(out)


def linearize(coords: np.ndarray, plan: BitPlan) -> Tuple[np.ndarray, np.ndarray]:
    """Vectorised bit gather. Returns (lo, hi) uint64 halves of each position."""
    coords = np.asarray(coords)
    M = coords.shape[1] if coords.ndim == 2 else 0
    lo = np.zeros(M, dtype=np.uint64)
    hi = np.zeros(M, dtype=np.uint64)
    one = np.uint64(1)
    for n in range(plan.nmodes):
        c = coords[n].astype(np.uint64)
        for g, q in enumerate(plan.positions[n]):
            b = (c >> np.uint64(g)) & one
            if q < 64:
                lo |= b << np.uint64(q)
            else:
                hi |= b << np.uint64(q - 64)
    return lo, hi


def delinearize(lo: np.ndarray, hi: np.ndarray, plan: BitPlan) -> np.ndarray:
    """Vectorised bit scatter back to coords uint32 [N, M]."""
    M = lo.shape[0]
    out = np.zeros((plan.nmodes, M), dtype=np.uint64)
    one = np.uint64(1)
    for n in range(plan.nmodes):
        for g, q in enumerate(plan.positions[n]):
            src = lo if q < 64 else hi
            b = (src >> np.uint64(q % 64)) & one
            out[n] |= b << np.uint64(g)
    return out.astype(np.uint32)


def check_coords(coords: np.ndarray, dims: Sequence[int]) -> None:
    for n, I in enumerate(dims):
        if coords.shape[1] and int(coords[n].max()) >= I:
            raise ValueError(f"coordinate out of range in mode {n}")


# ---------------------------------------------------------------------------
# ordering and the encoded tensor
# ---------------------------------------------------------------------------

def alto_order(lo: np.ndarray, hi: np.ndarray) -> np.ndarray:
    """Permutation that sorts by line position; ties keep input order."""
    M = lo.shape[0]
    return np.lexsort((np.arange(M), lo, hi))


@dataclasses.dataclass
class AltoTensor:
    plan: BitPlan
    lo: np.ndarray        # sorted positions, low 64 bits
    hi: np.ndarray        # sorted positions, high 64 bits
    vals: np.ndarray      # values in ALTO order (float32, as given)
    perm: np.ndarray      # input index of each ordered nonzero

    @property
    def nnz(self) -> int:
        return int(self.lo.shape[0])


def encode(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int]) -> AltoTensor:
    """Linearize then order (the two stages of Section III-A)."""
    plan = bit_plan(dims)
    if plan.nbits > 128:
        raise ValueError("more than 128 index bits")
    check_coords(coords, dims)
    lo, hi = linearize(coords, plan)
    perm = alto_order(lo, hi)
    return AltoTensor(plan, lo[perm], hi[perm], np.asarray(vals)[perm], perm)


def key_width_words(nbits: int) -> int:
    """64-bit words per position: 1 up to 64 bits, 2 up to 128 (Section V-A)."""
    return 1 if nbits <= 64 else 2


# ---------------------------------------------------------------------------
# Section IV-A: balanced line segments and their mode intervals
# ---------------------------------------------------------------------------

def segment_starts(M: int, L: int) -> np.ndarray:
    return np.array([(l * M) // L for l in range(L + 1)], dtype=np.uint64)


def partition(t: AltoTensor, L: int) -> Tuple[np.ndarray, np.ndarray]:
    """Start offsets [L+1] and closed mode intervals [L, N, 2] of each segment."""
    M = t.nnz
    N = t.plan.nmodes
    starts = segment_starts(M, L)
    coords = delinearize(t.lo, t.hi, t.plan)
    iv = np.empty((L, N, 2), dtype=np.uint32)
    for l in range(L):
        a, b = int(starts[l]), int(starts[l + 1])
        for n in range(N):
            if b > a:
                seg = coords[n, a:b]
                iv[l, n, 0] = seg.min()
                iv[l, n, 1] = seg.max()
            else:
                iv[l, n, 0] = EMPTY_LO
                iv[l, n, 1] = 0
    return starts, iv


def fiber_reuse(M: int, dims: Sequence[int]) -> List[float]:
    """Average nonzeros per fiber of each mode: M / I_n (Section IV-B)."""
    return [M / float(I) for I in dims]


def reuse_class(r: float) -> str:
    """High above 8, medium from 5 to 8, limited below (Section V-A)."""
    if r > 8:
        return "high"
    if r >= 5:
        return "medium"
    return "limited"


# ---------------------------------------------------------------------------
# Eq. 1-3: storage
# ---------------------------------------------------------------------------

def storage_bits_alto(dims: Sequence[int], M: int) -> int:
    """Eq. 1: M * sum_n log2 I_n bits (log2 read as bits per mode)."""
    return M * sum(mode_bits(I) for I in dims)


def coo_over_alto(dims: Sequence[int], word_bits: int) -> float:
    """Eq. 2: metadata ratio COO / ALTO with word size W_b."""
    b = [mode_bits(I) for I in dims]
    num = sum(-(-x // word_bits) for x in b)
    den = -(-sum(b) // word_bits)
    return num / den


def storage_bits_sfc(dims: Sequence[int], M: int) -> int:
    """Eq. 3: M * N * max_n log2 I_n bits for a Z-Morton style curve."""
    return M * len(dims) * max(mode_bits(I) for I in dims)


# ---------------------------------------------------------------------------
# MTTKRP: definition (Alg. 1 MTTKRP line, Alg. 3) and the dense check
# ---------------------------------------------------------------------------

def mttkrp(coords: np.ndarray, vals: np.ndarray, factors: Sequence[np.ndarray],
           mode: int) -> np.ndarray:
    """M(i,:) = sum over nonzeros x with i_mode(x) = i of v_x * prod_{m!=mode} A_m(i_m(x),:).

    fp64 from the given (float32 or float64) factors; duplicate coordinates are
    summed, each as its own term.
    """
    N = len(factors)
    R = factors[0].shape[1]
    I = factors[mode].shape[0]
    out = np.zeros((I, R), dtype=np.float64)
    M = coords.shape[1]
    step = 1 << 20
    for a in range(0, M, step):
        b = min(M, a + step)
        t = np.asarray(vals[a:b], dtype=np.float64)[:, None] * np.ones((1, R))
        for m in range(N):
            if m != mode:
                t = t * np.asarray(factors[m], dtype=np.float64)[coords[m, a:b].astype(np.int64)]
        np.add.at(out, coords[mode, a:b].astype(np.int64), t)
    return out


# ---------------------------------------------------------------------------
# Alg. 4, output-oriented branch: the stored order pos_out and the traversal
# ---------------------------------------------------------------------------

def pos_out(t: AltoTensor, L: int, mode: int) -> np.ndarray:
    """Ordered positions [M] (int64): inside every line segment l of L
    (Section IV-A), the segment's positions by increasing coordinate of
    `mode`, ties in line order (a stable sort per segment)."""
    M = t.nnz
    coords = delinearize(t.lo, t.hi, t.plan)
    starts = segment_starts(M, L)
    out = np.empty(M, dtype=np.int64)
    for l in range(L):
        a, b = int(starts[l]), int(starts[l + 1])
        out[a:b] = a + np.argsort(coords[mode, a:b], kind="stable")
    return out


def mttkrp_output_oriented(t: AltoTensor, factors: Sequence[np.ndarray], mode: int,
                           L: int) -> Tuple[np.ndarray, int, int]:
    """Alg. 4 with output-oriented traversal, segments taken one after the
    other: each segment visits its nonzeros in pos_out order, sums the
    contribution v * prod_{m != mode} A_m(i_m, :) of consecutive nonzeros with
    the same output row, and adds the sum to the output when the row changes
    (or the segment ends). Returns (M fp64, number of row updates, number of
    those updates that go to a boundary row, i.e. a row that another segment
    also updates)."""
    N = len(factors)
    R = factors[0].shape[1]
    out = np.zeros((factors[mode].shape[0], R), dtype=np.float64)
    coords = delinearize(t.lo, t.hi, t.plan)
    order = pos_out(t, L, mode)
    starts = segment_starts(t.nnz, L)
    F = [np.asarray(A, dtype=np.float64) for A in factors]
    owners = {}
    for l in range(L):
        a, b = int(starts[l]), int(starts[l + 1])
        for i in set(coords[mode, a:b].tolist()):
            owners[i] = owners.get(i, 0) + 1
    updates = boundary = 0
    for l in range(L):
        a, b = int(starts[l]), int(starts[l + 1])
        row, acc = None, None
        for k in range(a, b):
            x = int(order[k])
            i = int(coords[mode, x])
            term = float(t.vals[x]) * np.ones(R)
            for m in range(N):
                if m != mode:
                    term = term * F[m][int(coords[m, x])]
            if i != row:
                if row is not None:
                    out[row] += acc
                    updates += 1
                    boundary += owners[row] > 1
                row, acc = i, term
            else:
                acc = acc + term
        if row is not None:
            out[row] += acc
            updates += 1
            boundary += owners[row] > 1
    return out, updates, boundary


def to_dense(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int]) -> np.ndarray:
    X = np.zeros(tuple(dims), dtype=np.float64)
    np.add.at(X, tuple(coords.astype(np.int64)), np.asarray(vals, dtype=np.float64))
    return X


def unfold(X: np.ndarray, n: int) -> np.ndarray:
    """Mode-n matricization X_(n): mode-n fibers as columns, the remaining
    indices in their natural order with the last one varying fastest."""
    return np.moveaxis(X, n, 0).reshape(X.shape[n], -1)


def khatri_rao(mats: Sequence[np.ndarray], rank: Optional[int] = None) -> np.ndarray:
    """Column-wise Kronecker product A1 (.) A2 (.) ... (first factor slowest);
    the product of no matrices is a single row of ones."""
    R = mats[0].shape[1] if mats else int(rank)
    K = np.ones((1, R), dtype=np.float64)
    for A in mats:
        A = np.asarray(A, dtype=np.float64)
        K = (K[:, None, :] * A[None, :, :]).reshape(-1, R)
    return K


def mttkrp_dense(X: np.ndarray, factors: Sequence[np.ndarray], mode: int) -> np.ndarray:
    """X_(n) (A^(1) (.) ... A^(n-1) (.) A^(n+1) ... (.) A^(N)), Alg. 1."""
    others = [factors[m] for m in range(X.ndim) if m != mode]
    return unfold(X, mode) @ khatri_rao(others, factors[mode].shape[1])


# ---------------------------------------------------------------------------
# CP-ALS, Alg. 1
# ---------------------------------------------------------------------------

def _solve_spd_or_pinv(V: np.ndarray, M: np.ndarray) -> np.ndarray:
    """A = M V^dagger; Cholesky when V is positive definite, else pinv."""
    try:
        L = np.linalg.cholesky(V)
        Y = np.linalg.solve(L, M.T)
        return np.linalg.solve(L.T, Y).T
    except np.linalg.LinAlgError:
        return M @ np.linalg.pinv(V)


def tensor_norm_sq(coords: np.ndarray, vals: np.ndarray) -> float:
    """||X||^2 of the tensor the COO entries describe: entries with the same
    coordinates add up into one cell (Section II-C, COO), then the cells are
    squared and summed."""
    if coords.shape[1] == 0:
        return 0.0
    coords = np.asarray(coords)
    # identify equal coordinates: one integer per nonzero (the coordinates
    # side by side) when they fit 64 bits, else the rows of coords.T
    widths = [max(int(c.max()), 1).bit_length() for c in coords]
    if sum(widths) <= 64:
        key = np.zeros(coords.shape[1], dtype=np.uint64)
        shift = 0
        for c, w in zip(coords, widths):
            key |= c.astype(np.uint64) << np.uint64(shift)
            shift += w
        _, inv = np.unique(key, return_inverse=True)
    else:
        _, inv = np.unique(coords.T, axis=0, return_inverse=True)
    cells = np.bincount(inv.ravel(), weights=np.asarray(vals, dtype=np.float64))
    return float(np.sum(cells * cells))


def cp_fit(normX2: float, lam: np.ndarray, factors: Sequence[np.ndarray],
           M_last: np.ndarray) -> float:
    """1 - ||X - X_hat|| / ||X|| from lambda, the Grams and the last MTTKRP."""
    R = lam.shape[0]
    G = np.ones((R, R))
    for A in factors:
        G *= A.T @ A
    norm_hat2 = float(lam @ G @ lam)
    inner = float(np.sum(lam * np.sum(M_last * factors[-1], axis=0)))
    resid2 = max(0.0, normX2 + norm_hat2 - 2.0 * inner)
    if normX2 <= 0.0:
        return 0.0
    return 1.0 - np.sqrt(resid2) / np.sqrt(normX2)


# Relative norm under which a column of an update counts as zero.
ZERO_COLUMN_REL = 1e-12


def cp_als_mode_update(coords: np.ndarray, vals: np.ndarray, A: List[np.ndarray], n: int,
                       mttkrp_fn=None) -> Tuple[np.ndarray, np.ndarray]:
    """One pass of the inner loop of Alg. 1 for mode n, updating A[n] in place:
    V = Hadamard product of the other Grams, M = MTTKRP, A^(n) = M V^dagger,
    lambda = column norms, A^(n) normalised. Returns (M, lambda)."""
    if mttkrp_fn is None:
        mttkrp_fn = mttkrp
    N = len(A)
    R = A[0].shape[1]
    V = np.ones((R, R))
    for m in range(N):
        if m != n:
            V *= A[m].T @ A[m]
    M = mttkrp_fn(coords, vals, A, n)
    An = _solve_spd_or_pinv(V, M)
    lam = np.sqrt(np.sum(An * An, axis=0))
    # a column of rounding noise (norm below 1e-12 of the largest) is a zero
    # column: lambda_r = 0 and the column is set to 0, not scaled up
    lam = np.where(lam > ZERO_COLUMN_REL * np.max(lam, initial=0.0), lam, 0.0)
    scale = np.where(lam > 0, 1.0 / np.where(lam > 0, lam, 1.0), 0.0)
    A[n] = An * scale
    return M, lam


@dataclasses.dataclass
class CPResult:
    factors: List[np.ndarray]
    lam: np.ndarray
    fits: List[float]


def cp_als(coords: np.ndarray, vals: np.ndarray, dims: Sequence[int],
           init: Sequence[np.ndarray], iters: int, tol: float = 0.0,
           mttkrp_fn=None) -> CPResult:
    """Alg. 1 in fp64. ``tol == 0`` runs exactly ``iters`` iterations; otherwise
    it stops after the first iteration whose fit changed by less than tol."""
    if mttkrp_fn is None:
        mttkrp_fn = mttkrp
    N = len(dims)
    A = [np.asarray(f, dtype=np.float64).copy() for f in init]
    R = A[0].shape[1]
    lam = np.ones(R)
    normX2 = tensor_norm_sq(coords, vals)
    fits: List[float] = []
    prev: Optional[float] = None
    for _ in range(iters):
        M = None
        for n in range(N):
            M, lam = cp_als_mode_update(coords, vals, A, n, mttkrp_fn)
        fit = cp_fit(normX2, lam, A, M)
        fits.append(fit)
        if tol > 0 and prev is not None and abs(fit - prev) < tol:
            break
        prev = fit
    return CPResult(A, lam, fits)


def reconstruct_dense(lam: np.ndarray, factors: Sequence[np.ndarray]) -> np.ndarray:
    """sum_r lambda_r a_r^(1) o ... o a_r^(N) as a dense array (tiny sizes)."""
    R = lam.shape[0]
    X = np.zeros(tuple(A.shape[0] for A in factors))
    for r in range(R):
        t = np.array(lam[r])
        for A in factors:
            t = np.multiply.outer(t, A[:, r])
        X += t
    return X


# ---------------------------------------------------------------------------
# error metric used by the parity tests
# ---------------------------------------------------------------------------

def row_relative_error(got: np.ndarray, ref: np.ndarray) -> Tuple[float, int]:
    """max_i ||got_i - ref_i||_inf / ||ref_i||_inf over rows with ref_i != 0,
    and the number of all-zero reference rows where ``got`` is not exactly 0."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    scale = np.max(np.abs(ref), axis=1)
    diff = np.max(np.abs(got - ref), axis=1)
    nz = scale > 0
    err = float(np.max(diff[nz] / scale[nz])) if np.any(nz) else 0.0
    bad_zero = int(np.count_nonzero(diff[~nz] != 0))
    return err, bad_zero
