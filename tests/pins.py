"""Checks that pin the CPU oracle to facts other than itself.

Each ``check_*`` function takes a loaded oracle library (``lib``) and raises AssertionError
when the oracle disagrees with what the paper or plain mathematics fixes.  The test suite
runs them against the real oracle, and against deliberately broken copies of it (mutation
tests) to show that a plausible mistake anywhere in the oracle fails at least one of them.

Independent formulations used here (none of them calls the oracle's own helpers):
  * Alg. 1 ("Scalar Input") and Alg. 2 ("Vector Input") of Sec. 3.1, restated in Python under
    the project's readings: the carry holds suffix sums of the last w-1 inputs, X1 holds prefix
    sums capped at w addends, and the new carry is the suffix of the block's last w-1 lanes.
  * closed forms (constant input, x_i = i, monotone input, w = 1, w = n, affine special cases),
  * the prefix-difference identity for invertible operators (Sec. 2.2, Sec. 5),
  * string-based k-mers and reverse complements, exhaustive over all 4^8 strings of length 8,
  * the multiplicative form of Wang's mix, an exhaustive bijection check, and an inverse,
  * string-based brute-force minimizers, exhaustive over short sequences,
  * structural facts of the paper's k=3, w=3 minimizer example (Fig. 2, Sec. 2.4).
"""

from __future__ import annotations

import itertools
import math
import os

import numpy as np

import oracle as O

M32 = 0xFFFFFFFF
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


# ------------------------------------------------------------------------------------------
# Python statements of the operators (independent of the C oracle)
# ------------------------------------------------------------------------------------------

def _i32(v):
    v &= M32
    return v - (1 << 32) if v >= (1 << 31) else v


PY_OPS = {
    "add_i32": (lambda a, b: _i32(a + b), 0),
    "min_i32": (lambda a, b: min(a, b), (1 << 31) - 1),
    "max_i32": (lambda a, b: max(a, b), -(1 << 31)),
    "xor_i32": (lambda a, b: _i32(a ^ b), 0),
    # (a1,b1) then (a2,b2): x -> a2*(a1*x+b1)+b2
    "affine_u32": (lambda l, r: ((r[0] * l[0]) & M32, (r[0] * l[1] + r[1]) & M32), (1, 0)),
    "add_f32": (lambda a, b: a + b, 0.0),
}


def alg1_scalar_input(op, xs, w):
    """Alg. 1: a vector Y of suffix sums of the last w-1 inputs; each new input is broadcast to
    the first w lanes and added on the right; lane 0 is the next output; shift left by one."""
    f, e = PY_OPS[op]
    n = len(xs)
    if n < w:
        return []
    Y = [e] * w
    for j in range(w - 1):                      # Y_j = x_j (+) ... (+) x_{w-2}
        acc = xs[j]
        for t in range(j + 1, w - 1):
            acc = f(acc, xs[t])
        Y[j] = acc
    out = []
    for i in range(w - 1, n):
        Y = [f(Y[j], xs[i]) for j in range(w)]  # Y <- Y (+) X, X = (x_i, ..., x_i)
        out.append(Y[0])
        Y = Y[1:] + [e]                          # Y <- Y <<< 1
    return out


def alg2_vector_input(op, xs, w, P):
    """Alg. 2 with blocks of P >= w inputs: X1 = prefix sums of the block capped at w addends,
    output lane j = carry_j (+) X1_j for j <= w-2 and X1_j otherwise; the new carry lane j is
    the suffix X_{P-w+1+j} (+) ... (+) X_{P-1}."""
    f, e = PY_OPS[op]
    n = len(xs)
    if n < w:
        return []
    assert P >= w
    carry = []
    for j in range(w - 1):
        acc = xs[j]
        for t in range(j + 1, w - 1):
            acc = f(acc, xs[t])
        carry.append(acc)
    out = []
    i = w - 1
    while i < n:
        X = [xs[i + j] if i + j < n else e for j in range(P)]
        X1 = []
        for j in range(P):
            acc = X[max(0, j - w + 1)]
            for t in range(max(0, j - w + 1) + 1, j + 1):
                acc = f(acc, X[t])
            X1.append(acc)
        for j in range(P):
            if i + j >= n:
                break
            out.append(f(carry[j], X1[j]) if j <= w - 2 else X1[j])
        new = []
        for j in range(w - 1):
            acc = X[P - w + 1 + j]
            for t in range(P - w + 2 + j, P):
                acc = f(acc, X[t])
            new.append(acc)
        carry = new
        i += P
    return out


def short_block_window_sums(op, xs, w, B):
    """Eq. 2 combined over blocks of B < w inputs (the reading behind the chunked minimizer kernel):
    window p = suffix of its first block from p, the totals of the whole blocks inside it, and the
    prefix of its last block up to p + w - 1, combined left to right."""
    f, _ = PY_OPS[op]
    assert B < w
    out = []
    for p in range(len(xs) - w + 1):
        q = p + w - 1
        bp, bq = p // B, q // B
        acc = xs[p]
        for t in range(p + 1, (bp + 1) * B):     # suffix of the first block
            acc = f(acc, xs[t])
        for b in range(bp + 1, bq):              # whole blocks
            tot = xs[b * B]
            for t in range(b * B + 1, (b + 1) * B):
                tot = f(tot, xs[t])
            acc = f(acc, tot)
        pre = xs[bq * B]                          # prefix of the last block
        for t in range(bq * B + 1, q + 1):
            pre = f(pre, xs[t])
        out.append(f(acc, pre))
    return out


def short_block_argmin(xs, w, B):
    """The same decomposition for the minimum with the position of its leftmost occurrence, with
    the chunked kernel's tie rules: prefix minima and the left-to-right combination take a later
    element only when strictly smaller, suffix minima keep the earlier one on ties."""
    out = []
    for p in range(len(xs) - w + 1):
        q = p + w - 1
        bp, bq = p // B, q // B
        sv, sp = xs[(bp + 1) * B - 1], (bp + 1) * B - 1
        for t in range((bp + 1) * B - 2, p - 1, -1):  # suffix scan, backwards, <= keeps the earlier
            if xs[t] <= sv:
                sv, sp = xs[t], t
        acc = (sv, sp)
        for b in range(bp + 1, bq):
            tv, tp = xs[b * B], b * B
            for t in range(b * B + 1, (b + 1) * B):
                if xs[t] < tv:
                    tv, tp = xs[t], t
            if tv < acc[0]:
                acc = (tv, tp)
        pv, pp = xs[bq * B], bq * B
        for t in range(bq * B + 1, q + 1):
            if xs[t] < pv:
                pv, pp = xs[t], t
        if pv < acc[0]:
            acc = (pv, pp)
        out.append(acc)
    return out


def check_eq2_short_blocks(lib, seed=3, nmax=40):
    """Eq. 2 (oracle) = the combination over blocks shorter than w, every operator (the affine
    maps are not commutative, so the order of the pieces matters), every B < w <= n; and for the
    minimum, the leftmost argmin of every window by brute force (few distinct values: many ties)."""
    rng = np.random.default_rng(seed)
    for op in PY_OPS:
        for n in (17, 23, nmax):
            xs = _rand_elems(op, n, rng)
            for w in range(2, n + 1):
                got = _from_oracle_output(op, O.sliding_sum(op, w, _to_oracle_input(op, xs), lib=lib))
                for B in (1, 2, 3, 5, 16):
                    if B >= w:
                        continue
                    ref = short_block_window_sums(op, xs, w, B)
                    if op == "add_f32":
                        for p, (a, b) in enumerate(zip(got, ref)):
                            assert _close_f(a, b, sum(abs(v) for v in xs[p:p + w])), (op, n, w, B, p)
                    else:
                        assert got == ref, (op, n, w, B)
    for trial in range(40):
        n = int(rng.integers(17, 90))
        xs = [int(v) for v in rng.integers(0, 4, size=n)]
        for w in (17, 18, 31, 32, 33, 50, 64, 65):
            if w > n:
                continue
            got = short_block_argmin(xs, w, 16)
            for p, (v, pos) in enumerate(got):
                seg = xs[p:p + w]
                assert v == min(seg) and pos == p + seg.index(min(seg)), (n, w, p)


def _rand_elems(op, n, rng):
    if op == "affine_u32":
        return [(int(a), int(b)) for a, b in rng.integers(0, 1 << 32, size=(n, 2), dtype=np.uint64)]
    if op == "add_f32":
        return [float(np.float32(v)) for v in rng.standard_normal(n)]
    return [int(v) for v in rng.integers(-(1 << 31), 1 << 31, size=n, dtype=np.int64)]


def _to_oracle_input(op, xs):
    if op == "affine_u32":
        return np.asarray(xs, dtype=np.uint64).astype(np.uint32)
    if op == "add_f32":
        return np.asarray(xs, dtype=np.float32)
    return np.asarray(xs, dtype=np.int64).astype(np.int32)


def _from_oracle_output(op, y):
    if op == "affine_u32":
        return [(int(a), int(b)) for a, b in y]
    if op == "add_f32":
        return [float(v) for v in y]
    return [int(v) for v in y]


def _close_f(a, b, xs_abs_window):
    return abs(a - b) <= 64 * 2.0 ** -53 * xs_abs_window + 1e-300


def check_eq2_vs_algorithms(lib, seed=1, nmax=11):
    """Eq. 2 (oracle) = Alg. 1 = Alg. 2 for every operator, every w <= n, several P."""
    rng = np.random.default_rng(seed)
    for op in PY_OPS:
        for n in range(0, nmax + 1):
            xs = _rand_elems(op, n, rng)
            for w in range(1, n + 1):
                got = _from_oracle_output(op, O.sliding_sum(op, w, _to_oracle_input(op, xs), lib=lib))
                assert len(got) == n - w + 1, (op, n, w)
                refs = [alg1_scalar_input(op, xs, w)] + [alg2_vector_input(op, xs, w, P) for P in (w, w + 1, 2 * w + 1)]
                for ref in refs:
                    assert len(ref) == len(got)
                    if op == "add_f32":
                        for p, (a, b) in enumerate(zip(got, ref)):
                            s = sum(abs(v) for v in xs[p:p + w])
                            assert _close_f(a, b, s), (op, n, w, p, a, b)
                    else:
                        assert got == ref, (op, n, w, got, ref)
            # n < w: nothing
            assert O.sliding_sum(op, n + 1, _to_oracle_input(op, xs), lib=lib).shape[0] == 0


def check_eq2_closed_forms(lib):
    """Closed forms of Eq. 2."""
    n = 200
    for w in (1, 2, 3, 7, 64, 200):
        # constant input, + mod 2^32
        c = 123456789
        y = O.sliding_sum("add_i32", w, np.full(n, c, dtype=np.int32), lib=lib)
        assert (y.astype(np.int64) & M32 == (w * c) & M32).all()
        # x_i = i, + : y_p = w p + w(w-1)/2
        y = O.sliding_sum("add_i32", w, np.arange(n, dtype=np.int32), lib=lib)
        p = np.arange(n - w + 1, dtype=np.int64)
        assert (y.astype(np.int64) == w * p + w * (w - 1) // 2).all()
        # monotone increasing input: min = first, max = last addend
        x = (np.arange(n, dtype=np.int64) * 3 - 100).astype(np.int32)
        assert (O.sliding_sum("min_i32", w, x, lib=lib) == x[: n - w + 1]).all()
        assert (O.sliding_sum("max_i32", w, x, lib=lib) == x[w - 1:]).all()
        # xor of a constant: c if w odd else 0
        y = O.sliding_sum("xor_i32", w, np.full(n, 0x5A5A5A5A, dtype=np.int32), lib=lib)
        assert (y == (0x5A5A5A5A if w % 2 else 0)).all()
    rng = np.random.default_rng(7)
    x = rng.integers(-(1 << 31), 1 << 31, size=50, dtype=np.int64).astype(np.int32)
    # w = 1: identity; w = n: total reduction
    for op in ("add_i32", "min_i32", "max_i32", "xor_i32"):
        assert (O.sliding_sum(op, 1, x, lib=lib) == x).all()
    tot = O.sliding_sum("add_i32", 50, x, lib=lib)
    assert tot.shape == (1,) and int(tot[0]) & M32 == int(x.astype(np.int64).sum()) & M32
    assert int(O.sliding_sum("min_i32", 50, x, lib=lib)[0]) == int(x.min())
    assert int(O.sliding_sum("max_i32", 50, x, lib=lib)[0]) == int(x.max())
    assert int(O.sliding_sum("xor_i32", 50, x, lib=lib)[0]) == int(np.bitwise_xor.reduce(x))
    # affine special cases
    b = rng.integers(0, 1 << 32, size=60, dtype=np.uint64)
    a = rng.integers(0, 1 << 32, size=60, dtype=np.uint64)
    for w in (1, 5, 60):
        ones = np.stack([np.ones(60, dtype=np.uint64), b], 1).astype(np.uint32)
        y = O.sliding_sum("affine_u32", w, ones, lib=lib)
        for pp in range(60 - w + 1):
            assert int(y[pp, 0]) == 1 and int(y[pp, 1]) == int(b[pp:pp + w].sum()) & M32
        zeros = np.stack([a, np.zeros(60, dtype=np.uint64)], 1).astype(np.uint32)
        y = O.sliding_sum("affine_u32", w, zeros, lib=lib)
        for pp in range(60 - w + 1):
            prod = 1
            for t in range(pp, pp + w):
                prod = (prod * int(a[t])) & M32
            assert int(y[pp, 0]) == prod and int(y[pp, 1]) == 0
    # affine semantics: y_p applied to z equals applying f_p first, then f_{p+1}, ...
    ab = np.stack([a, b], 1).astype(np.uint32)
    for w in (2, 3, 9):
        y = O.sliding_sum("affine_u32", w, ab, lib=lib)
        for pp in (0, 17, 60 - w):
            for z in (0, 1, 987654321):
                v = z
                for t in range(pp, pp + w):
                    v = (int(a[t]) * v + int(b[t])) & M32
                assert (int(y[pp, 0]) * z + int(y[pp, 1])) & M32 == v
    # fp32 add: against math.fsum (exactly rounded), within fp64 accumulation error
    xf = np.random.default_rng(3).standard_normal(300).astype(np.float32)
    for w in (1, 4, 33, 300):
        y = O.sliding_sum("add_f32", w, xf, lib=lib)
        for pp in range(0, 300 - w + 1, 7):
            ref = math.fsum(float(v) for v in xf[pp:pp + w])
            assert _close_f(float(y[pp]), ref, float(np.abs(xf[pp:pp + w].astype(np.float64)).sum()))


def check_prefix_difference(lib):
    """Invertible operators: y_p = S_{p+w-1} (-) S_{p-1} with prefix sums S (Sec. 2.2, Sec. 5)."""
    rng = np.random.default_rng(11)
    x = rng.integers(-(1 << 31), 1 << 31, size=5000, dtype=np.int64).astype(np.int32)
    xu = x.view(np.uint32).astype(np.uint64)
    z = np.zeros(1, dtype=np.uint64)
    S = np.concatenate([z, np.cumsum(xu) & np.uint64(M32)])
    X = np.concatenate([z, np.bitwise_xor.accumulate(xu)])
    for w in (1, 2, 16, 100, 1024):
        y = O.sliding_sum("add_i32", w, x, lib=lib).view(np.uint32).astype(np.uint64)
        assert (y == (S[w:] - S[: 5000 - w + 1]) & np.uint64(M32)).all()
        y = O.sliding_sum("xor_i32", w, x, lib=lib).view(np.uint32).astype(np.uint64)
        assert (y == X[w:] ^ X[: 5000 - w + 1]).all()


def check_sampled_matches_full(lib):
    rng = np.random.default_rng(5)
    for op in ("add_i32", "min_i32", "affine_u32", "add_f32"):
        n = 3000
        x = _to_oracle_input(op, _rand_elems(op, n, rng))
        for w in (1, 13, 256):
            full = O.sliding_sum(op, w, x, lib=lib)
            idx = np.array([0, 1, 77, n - w], dtype=np.uint64)
            assert (O.sliding_sum_at(op, w, x, idx, lib=lib) == full[idx.astype(np.int64)]).all()


# ------------------------------------------------------------------------------------------
# k-mers and hash
# ------------------------------------------------------------------------------------------

_COMP = str.maketrans("ACGT", "TGCA")
_DIG = str.maketrans("ACGT", "0123")


def pack_string(s: str) -> np.ndarray:
    codes = np.frombuffer(s.translate(_DIG).encode(), dtype=np.uint8) - ord("0")
    nb = (len(s) + 3) // 4
    c = np.zeros(nb * 4, dtype=np.uint8)
    c[: len(s)] = codes
    c = c.reshape(nb, 4)
    return (c[:, 0] | (c[:, 1] << 2) | (c[:, 2] << 4) | (c[:, 3] << 6)).astype(np.uint8)


def revcomp(s: str) -> str:
    return s.translate(_COMP)[::-1]


def kval(s: str) -> int:
    return int(s.translate(_DIG), 4) if s else 0


def wang_mult_form(x: int, bits: int) -> int:
    """Wang's mix written with the multipliers its steps stand for (published comments):
    (key << 21) - key - 1, key * 265, key * 21, key * (1 + 2^31); each truncated to ``bits``."""
    m = (1 << bits) - 1
    x &= m
    x = (x * ((1 << 21) - 1) - 1) & m
    x ^= x >> 24
    x = (x * 265) & m
    x ^= x >> 14
    x = (x * 21) & m
    x ^= x >> 28
    x = (x * ((1 << 31) + 1)) & m
    return x


def check_kmers_exhaustive8(lib):
    """All 4^8 strings of length 8 (concatenated), every k-mer kind, against string arithmetic."""
    strs = ["".join(t) for t in itertools.product("ACGT", repeat=8)]
    S = "".join(strs)
    seq = pack_string(S)
    n = len(S)
    for k in (8, 3, 1):
        fwd = O.kmers(seq, n, k, "fwd", lib=lib)
        rc = O.kmers(seq, n, k, "rc", lib=lib)
        can = O.kmers(seq, n, k, "canonical", lib=lib)
        hsh = O.kmers(seq, n, k, "hash", lib=lib)
        step = 8 if k == 8 else 997
        for i in range(0, n - k + 1, step):
            sub = S[i:i + k]
            f, r = kval(sub), kval(revcomp(sub))
            assert int(fwd[i]) == f and int(rc[i]) == r and int(can[i]) == min(f, r), (k, i, sub)
            assert int(hsh[i]) == wang_mult_form(min(f, r), 2 * k)


def check_kmer_symmetries(lib):
    rng = np.random.default_rng(2)
    S = "".join(rng.choice(list("ACGT"), size=777))
    R = revcomp(S)
    n = len(S)
    for k in (1, 5, 15, 19, 32):
        m = n - k + 1
        rc = O.kmers(pack_string(S), n, k, "rc", lib=lib)
        fwd_r = O.kmers(pack_string(R), n, k, "fwd", lib=lib)
        assert (rc == fwd_r[::-1]).all()  # rc of k-mer i = forward k-mer m-1-i of revcomp(S)
        can = O.kmers(pack_string(S), n, k, "canonical", lib=lib)
        can_r = O.kmers(pack_string(R), n, k, "canonical", lib=lib)
        assert (can == can_r[::-1]).all()
        assert m == can.shape[0]
        for i in (0, 1, m // 2, m - 1):
            assert int(O.kmers(pack_string(S), n, k, "fwd", lib=lib)[i]) == kval(S[i:i + k])


def check_hash(lib, exhaustive_bits=(2, 4, 10, 16, 22)):
    rng = np.random.default_rng(9)
    for bits in (2, 8, 30, 38, 62, 64):
        m = (1 << bits) - 1
        for x in rng.integers(0, 1 << 63, size=200, dtype=np.uint64):
            x = int(x) & m
            h = O.hash64(x, bits, lib=lib)
            assert h == wang_mult_form(x, bits), (bits, x)
            assert O.hash64_inv(h, bits, lib=lib) == x
    for bits in exhaustive_bits:
        assert O.hash_is_bijection(bits, lib=lib)


# ------------------------------------------------------------------------------------------
# Minimizers
# ------------------------------------------------------------------------------------------

def brute_minimizers(S: str, k: int, w: int, mode: str):
    """String-based minimizers: split at 'N', per stretch take each window of w k-mers, the
    least (key, position), and store consecutive repeats once."""
    out = []
    a = 0
    n = len(S)
    while a < n:
        if S[a] == "N":
            a += 1
            continue
        b = a
        while b < n and S[b] != "N":
            b += 1
        run = S[a:b]
        keys = []
        for i in range(len(run) - k + 1):
            sub = run[i:i + k]
            f, r = kval(sub), kval(revcomp(sub))
            if mode == "fwd":
                keys.append(f)
            elif mode == "canonical":
                keys.append(min(f, r))
            else:
                keys.append(wang_mult_form(min(f, r), 2 * k))
        last = None
        for p in range(len(keys) - w + 1):
            best = min(range(p, p + w), key=lambda j: (keys[j], j))
            if best != last:
                out.append((keys[best], a + best))
            last = best
        a = b
    return out


def _oracle_pairs(lib, S, k, w, mode, deque=False):
    seq = pack_string(S.replace("N", "A"))
    iv = []
    i = 0
    while i < len(S):
        if S[i] == "N":
            j = i
            while j < len(S) and S[j] == "N":
                j += 1
            iv.append((i, j))
            i = j
        else:
            i += 1
    h, p = O.minimizers(seq, len(S), k, w, mode, nblocks=np.array(iv, dtype=np.int64).reshape(-1, 2),
                        deque=deque, lib=lib)
    return list(zip((int(v) for v in h), (int(v) for v in p)))


def check_minimizers_bruteforce(lib):
    """Exhaustive short sequences (fwd keys) plus random ones with N-blocks (all key modes)."""
    for n in range(1, 8):
        for t in itertools.product("ACGT", repeat=n):
            S = "".join(t)
            for k in (1, 2, 3):
                for w in (1, 2, 3, 4):
                    if k + w - 1 > n + 1:
                        continue
                    exp = brute_minimizers(S, k, w, "fwd")
                    assert _oracle_pairs(lib, S, k, w, "fwd") == exp, (S, k, w)
    rng = np.random.default_rng(4)
    for trial in range(60):
        n = int(rng.integers(1, 90))
        S = list(rng.choice(list("ACGT"), size=n))
        for _ in range(int(rng.integers(0, 4))):
            s = int(rng.integers(0, n))
            S[s:s + int(rng.integers(1, 6))] = ["N"] * len(S[s:s + int(rng.integers(1, 6))])
        S = "".join(S)[:n]
        for mode in ("fwd", "canonical", "hash"):
            for k, w in ((1, 1), (3, 3), (4, 2), (5, 7), (15, 10)):
                exp = brute_minimizers(S, k, w, mode)
                assert _oracle_pairs(lib, S, k, w, mode) == exp, (S, k, w, mode)
                assert _oracle_pairs(lib, S, k, w, mode, deque=True) == exp, (S, k, w, mode, "deque")


def check_minimizer_invariants(lib):
    """On a 20 kb random sequence: naive = deque; every pick is the least key of some window;
    positions strictly increase; every window's least key is among the picks; density near
    2/(w+1) picks per k-mer (Roberts et al. expectation for random sequences)."""
    rng = np.random.default_rng(8)
    S = "".join(rng.choice(list("ACGT"), size=20000))
    seq = pack_string(S)
    n = len(S)
    for k, w in ((15, 10), (19, 10), (15, 50), (5, 4)):
        h, p = O.minimizers(seq, n, k, w, "hash", lib=lib)
        h2, p2 = O.minimizers(seq, n, k, w, "hash", deque=True, lib=lib)
        assert (h == h2).all() and (p == p2).all()
        keys = O.kmers(seq, n, k, "hash", lib=lib)
        assert (np.diff(p.astype(np.int64)) > 0).all()
        assert (keys[p.astype(np.int64)] == h).all()
        picked = set(int(v) for v in p)
        nw = n - k - w + 2
        for q in range(0, nw, 37):
            win = keys[q:q + w]
            j = q + int(np.argmin(win))  # argmin returns the first (leftmost) minimum
            assert j in picked
        dens = len(p) / (n - k + 1)
        assert abs(dens - 2.0 / (w + 1)) < 0.25 * 2.0 / (w + 1), (k, w, dens)


def check_fig2_example(lib):
    """Structural facts of the paper's k=3, w=3 example (Fig. 2, Sec. 2.4) on a sequence built
    to satisfy them (the figure's own sequence is not in the text): four windows p = 0..3;
    windows 1 and 2 share the pick ('CTT', 2); stored positions are exactly {0, 2, 5}."""
    path = os.path.join(GOLDEN, "fig2_minimizer_example.txt")
    fields = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                key, val = line.split("=", 1)
                fields[key.strip()] = val.strip()
    S = fields["sequence"]
    k, w = int(fields["k"]), int(fields["w"])
    want_pos = [int(v) for v in fields["stored_positions"].split(",")]
    shared_seed, shared_pos = fields["shared_pick"].split(",")
    pairs = _oracle_pairs(lib, S, k, w, "fwd")
    assert len(S) - k - w + 2 == int(fields["windows"])
    assert [p for _, p in pairs] == want_pos
    assert (kval(shared_seed), int(shared_pos)) in pairs
    for key, pos in pairs:
        assert key == kval(S[pos:pos + k])


def check_batch_and_keys(lib):
    rng = np.random.default_rng(12)
    lens = rng.integers(1, 60, size=40)
    S = "".join(rng.choice(list("ACGT"), size=int(lens.sum())))
    offs = np.concatenate([[0], np.cumsum(lens)])
    h, p, po = O.minimizers_batch(pack_string(S), offs, 5, 4, "hash", lib=lib)
    cur = 0
    for r in range(len(lens)):
        exp = brute_minimizers(S[offs[r]:offs[r + 1]], 5, 4, "hash")
        got = list(zip((int(v) for v in h[po[r]:po[r + 1]]), (int(v) for v in p[po[r]:po[r + 1]])))
        assert int(po[r]) == cur and got == exp
        cur += len(exp)
    assert int(po[-1]) == cur == len(h)
    keys = rng.integers(0, 1 << 30, size=500, dtype=np.uint64)
    keys[100:140] = 5  # a run of equal keys: the leftmost must win
    keys[300:330] = rng.integers(0, 3, size=30)  # few distinct values: ties everywhere
    for w in (1, 2, 4, 10, 17):
        exp = []
        last = None
        for q in range(500 - w + 1):
            j = min(range(q, q + w), key=lambda t: (int(keys[t]), t))
            if j != last:
                exp.append((int(keys[j]), j))
            last = j
        for deque in (False, True):  # the naive scan ("Array") and the queue ("Dequeue") of Sec. 4
            kh, kp = O.minimizers_from_keys(keys, w, deque=deque, lib=lib)
            assert list(zip((int(v) for v in kh), (int(v) for v in kp))) == exp, (w, deque)


def check_table(lib):
    rng = np.random.default_rng(13)
    for hash_bits, bucket_bits in ((30, 12), (20, 20), (38, 16), (8, 0)):
        m = 3000
        h = rng.integers(0, 1 << hash_bits, size=m, dtype=np.uint64)
        h[::5] = h[0]
        p = np.sort(rng.choice(1 << 31, size=m, replace=False)).astype(np.uint32)
        sh, sp, off = O.kmer_table(h, p, hash_bits, bucket_bits, lib=lib)
        assert sorted(zip(h.tolist(), p.tolist())) == list(zip(sh.tolist(), sp.tolist()))
        shift = hash_bits - bucket_bits
        cnt = np.bincount((h >> np.uint64(shift)).astype(np.int64), minlength=1 << bucket_bits)
        assert (np.diff(off.astype(np.int64)) == cnt).all() and int(off[0]) == 0 and int(off[-1]) == m
        for i in rng.integers(0, m, size=50):
            b = int(h[i]) >> shift
            lo, hi = int(off[b]), int(off[b + 1])
            assert (int(h[i]), int(p[i])) in set(zip(sh[lo:hi].tolist(), sp[lo:hi].tolist()))


def check_seed_hits(lib):
    """Seed hits against a brute force over a dict: query i hits every reference position whose
    seed hash equals its own, seeds with more than max_occ hits skipped; pairs in query order,
    positions ascending."""
    rng = np.random.default_rng(17)
    for m, nq, hi, max_occ in ((0, 5, 4, 0), (1, 1, 1, 0), (400, 120, 30, 0), (400, 120, 30, 15), (3000, 500, 1 << 38, 0),
                               (2000, 300, 8, 250)):
        h = rng.integers(0, hi, size=m, dtype=np.uint64)
        p = rng.permutation(1 << 20)[:m].astype(np.uint32)
        q = rng.integers(0, hi + 2, size=nq, dtype=np.uint64)
        if m:
            q[::3] = h[rng.integers(0, m, size=q[::3].size)]
        table = {}
        for hv, pv in zip(h.tolist(), p.tolist()):
            table.setdefault(hv, []).append(pv)
        exp_cnt, exp_pairs = [], []
        for i, qv in enumerate(q.tolist()):
            hits = sorted(table.get(qv, []))
            exp_cnt.append(len(hits))
            if max_occ == 0 or len(hits) <= max_occ:
                exp_pairs += [(i, x) for x in hits]
        cnt, hq, hp = O.seed_hits(h, p, q, max_occ, lib=lib)
        assert cnt.tolist() == exp_cnt
        assert list(zip(hq.tolist(), hp.tolist())) == exp_pairs


def check_strands(lib):
    """Strand of canonical picks against strings: 1 iff the reverse complement is smaller."""
    rng = np.random.default_rng(23)
    comp = {"A": "T", "C": "G", "G": "C", "T": "A"}
    for k in (1, 2, 5, 6, 15, 19, 32):
        n = 300
        codes = rng.integers(0, 4, size=n)
        st = "".join("ACGT"[c] for c in codes)
        packed = pack_string(st)
        pos = rng.integers(0, n - k + 1, size=60).astype(np.uint32)
        pos = np.concatenate([pos, [n - k + 1, n]]).astype(np.uint32)  # two outside the sequence
        got = O.strands(packed, n, k, pos, lib=lib)
        for i, p in enumerate(pos.tolist()):
            if p + k > n:
                assert got[i] == 255
                continue
            f = st[p:p + k]
            r = "".join(comp[c] for c in reversed(f))
            assert got[i] == (1 if r < f else 0), (k, p, f, r)
    # a batch: read-local positions
    lens = [40, 0, 25, 60]
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    codes = rng.integers(0, 4, size=int(offs[-1]))
    packed = pack_string("".join("ACGT"[c] for c in codes))
    k = 7
    pos, po = [], [0]
    for L in lens:
        q = list(range(0, max(L - k + 1, 0), 3))
        pos += q
        po.append(po[-1] + len(q))
    got = O.strands(packed, int(offs[-1]), k, np.array(pos, np.uint32), offs, np.array(po, np.uint64), lib=lib)
    st = "".join("ACGT"[c] for c in codes)
    for r in range(len(lens)):
        for i in range(po[r], po[r + 1]):
            f = st[offs[r] + pos[i]:offs[r] + pos[i] + k]
            rc = "".join(comp[c] for c in reversed(f))
            assert got[i] == (1 if rc < f else 0)


ALL_CHECKS = [
    check_eq2_vs_algorithms,
    check_eq2_short_blocks,
    check_eq2_closed_forms,
    check_prefix_difference,
    check_sampled_matches_full,
    check_kmers_exhaustive8,
    check_kmer_symmetries,
    check_hash,
    check_minimizers_bruteforce,
    check_minimizer_invariants,
    check_fig2_example,
    check_batch_and_keys,
    check_table,
    check_seed_hits,
    check_strands,
]
