#!/usr/bin/env python3
"""Generates ``bitsliced_sbox.cuh``: the AES S-box (FIPS-197 sec. 5.1.1) as a
boolean circuit of AND / XOR gates, for bitsliced AES on the GPU.

Derivation (no table is copied; everything follows from the field):

* The S-box is S(a) = A * a^-1 + 0x63 in GF(2^8) = GF(2)[x]/(x^8 + x^4 + x^3 +
  x + 1), with A the FIPS-197 affine matrix and 0^-1 = 0.
* Inversion is done in an isomorphic tower field GF(((2^2)^2)^2):
    GF(4)   = GF(2)[w]/(w^2 + w + 1)
    GF(16)  = GF(4)[z]/(z^2 + z + nu)       (nu chosen so this is irreducible)
    GF(256) = GF(16)[y]/(y^2 + y + lam)     (lam chosen likewise)
  For X = x1*y + x0 over a subfield with y^2 = y + lam, the product
  X * (x1*y + x1 + x0) is the subfield element D = lam*x1^2 + x1*x0 + x0^2,
  so X^-1 = D^-1 * (x1*y + x1 + x0); D = 0 only for X = 0, and the same
  formula then gives 0.  GF(16) inversion uses the same identity one level
  down, and in GF(4) the inverse is the square.
* The isomorphism maps the AES basis {1, x, ..., x^7} to the powers of a root
  of the AES polynomial found in the tower field; the input change of basis
  M and the output map A * M^-1 are 8 x 8 matrices over GF(2), turned into
  XOR networks with a greedy shared-pair heuristic (Paar).
* The additive constant 0x63 is not in the circuit: the caller folds it into
  the next round key (MixColumns maps a column of equal bytes c to itself
  since 2 + 3 + 1 + 1 = 1 in GF(2^8)).

The generated circuit is checked against the S-box computed here from its
definition on all 256 inputs before anything is written.

Usage: python gen_bitsliced_sbox.py [output path]
"""
import argparse
import itertools
import os
import random
import sys

AES_POLY = 0x11B


# ---------------------------------------------------------------------------
# Reference arithmetic (plain integers) for the check
# ---------------------------------------------------------------------------
def aes_mul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        if a & 0x100:
            a ^= AES_POLY
        b >>= 1
    return r


def aes_inv(a):
    if a == 0:
        return 0
    r = 1
    for _ in range(254):  # a^254 = a^-1 in a field of 256 elements
        r = aes_mul(r, a)
    return r


def affine(b):
    """FIPS-197 affine map without its constant: bit i of the result is
    b_i + b_{i+4} + b_{i+5} + b_{i+6} + b_{i+7} (indices mod 8)."""
    r = 0
    for i in range(8):
        bit = 0
        for k in (0, 4, 5, 6, 7):
            bit ^= (b >> ((i + k) % 8)) & 1
        r |= bit << i
    return r


def sbox(a):
    return affine(aes_inv(a)) ^ 0x63


# ---------------------------------------------------------------------------
# Tower field on integers (for finding the isomorphism)
# Element of GF(4): 2 bits (bit1 = coefficient of w).  GF(16): 4 bits (high
# pair = coefficient of z).  GF(256): 8 bits (high nibble = coefficient of y).
# ---------------------------------------------------------------------------
def g4_mul(a, b):
    a1, a0, b1, b0 = a >> 1, a & 1, b >> 1, b & 1
    hi = (a1 & b1) ^ (a1 & b0) ^ (a0 & b1)
    lo = (a1 & b1) ^ (a0 & b0)
    return (hi << 1) | lo


def g16_mul(a, b, nu):
    a1, a0, b1, b0 = a >> 2, a & 3, b >> 2, b & 3
    p11 = g4_mul(a1, b1)
    hi = p11 ^ g4_mul(a1, b0) ^ g4_mul(a0, b1)
    lo = g4_mul(p11, nu) ^ g4_mul(a0, b0)
    return (hi << 2) | lo


def g256_mul(a, b, nu, lam):
    a1, a0, b1, b0 = a >> 4, a & 15, b >> 4, b & 15
    p11 = g16_mul(a1, b1, nu)
    hi = p11 ^ g16_mul(a1, b0, nu) ^ g16_mul(a0, b1, nu)
    lo = g16_mul(p11, lam, nu) ^ g16_mul(a0, b0, nu)
    return (hi << 4) | lo


def irreducible_over(n_bits, mul, c):
    """y^2 + y + c has no root in the field of 2^n_bits elements."""
    return all(mul(t, t) ^ t ^ c for t in range(1 << n_bits))


# Tower parameters and the root of the AES polynomial used for the change of
# basis.  Every valid choice gives a correct circuit; this one (found with
# --search over nu, lambda, the eight roots and the tie-breaking seed of the
# XOR-sharing heuristic) gives the fewest gates: 36 AND + 93 XOR.
NU, LAM, BETA, SEED = 3, 11, 92, 2


def valid_params(nu, lam):
    return irreducible_over(2, g4_mul, nu) and irreducible_over(4, lambda a, b: g16_mul(a, b, nu), lam)


def aes_roots(nu, lam):
    """Roots beta of the AES polynomial in the tower field whose powers
    beta^0..beta^7 form a basis; the columns beta^i give tower(a) = M aes(a)."""
    def mul(a, b):
        return g256_mul(a, b, nu, lam)

    def power(b, e):
        r = 1
        for _ in range(e):
            r = mul(r, b)
        return r

    out = {}
    for beta in range(2, 256):
        # x^8 + x^4 + x^3 + x + 1 at beta
        if power(beta, 8) ^ power(beta, 4) ^ power(beta, 3) ^ beta ^ 1 == 0:
            cols = [power(beta, i) for i in range(8)]
            if rank(cols) == 8:
                out[beta] = cols
    return out


def rank(cols):
    rows = list(cols)
    r = 0
    for bit in range(8):
        piv = next((i for i in range(r, len(rows)) if (rows[i] >> bit) & 1), None)
        if piv is None:
            continue
        rows[r], rows[piv] = rows[piv], rows[r]
        for i in range(len(rows)):
            if i != r and (rows[i] >> bit) & 1:
                rows[i] ^= rows[r]
        r += 1
    return r


def mat_apply(cols, v):
    r = 0
    for i in range(8):
        if (v >> i) & 1:
            r ^= cols[i]
    return r


def mat_inverse(cols):
    """Inverse of the linear map given by columns (as a column list)."""
    inv = [0] * 8
    for i in range(8):
        # find v with M v = e_i by brute force (256 candidates)
        inv[i] = next(v for v in range(256) if mat_apply(cols, v) == (1 << i))
    return inv


# ---------------------------------------------------------------------------
# Circuit builder
# ---------------------------------------------------------------------------
class Circuit:
    def __init__(self, n_in):
        self.gates = []  # (op, a, b): op in '^', '&'; wires are ints
        self.n_in = n_in

    def new(self, op, a, b):
        self.gates.append((op, a, b))
        return self.n_in + len(self.gates) - 1

    def xor(self, a, b):
        if a is None:
            return b
        if b is None:
            return a
        return self.new("^", a, b)

    def and_(self, a, b):
        return self.new("&", a, b)

    def xor_many(self, ws):
        acc = None
        for w in ws:
            acc = self.xor(acc, w)
        return acc


def linear_network(circ, in_wires, rows_masks, rng):
    """XOR network computing outputs o_r = XOR of in_wires[i] for i in
    rows_masks[r]: repeatedly adds the XOR of the pair of wires shared by the
    most outputs (Paar's greedy heuristic; ties broken by rng)."""
    wires = list(in_wires)
    rows = [set(i for i in range(len(in_wires)) if (m >> i) & 1) for m in rows_masks]
    while True:
        cand, best_n = [], 1
        for i, j in itertools.combinations(range(len(wires)), 2):
            n = sum(1 for r in rows if i in r and j in r)
            if n > best_n:
                cand, best_n = [(i, j)], n
            elif n == best_n and n > 1:
                cand.append((i, j))
        if not cand:
            break
        i, j = rng.choice(cand)
        wires.append(circ.xor(wires[i], wires[j]))
        k = len(wires) - 1
        for r in rows:
            if i in r and j in r:
                r.discard(i)
                r.discard(j)
                r.add(k)
    return [circ.xor_many([wires[i] for i in sorted(r)]) if r else None for r in rows]


def forms9(e):
    """The 9 linear forms of a GF(16) element (bits l0, l1, h0, h1 as masks)
    whose pairwise products give a GF(16) product: per GF(4) product u*v the
    operands u1, u0, u1 + u0; and the GF(16) product multiplies the pairs
    (a1, b1), (a0, b0) and (a1 + a0, b1 + b0)."""
    l0, l1, h0, h1 = e
    return [h1, h0, h1 ^ h0, l1, l0, l1 ^ l0, h1 ^ l1, h0 ^ l0, h1 ^ h0 ^ l1 ^ l0]


def forms3(e):
    """The 3 forms of a GF(4) element (bits (b0, b1) as masks)."""
    b0, b1 = e
    return [b1, b0, b1 ^ b0]


def solve_gf2(columns, target):
    """Coefficients c (mask over columns) with XOR of the selected columns ==
    target; columns and target are ints over the same bit positions."""
    rows = []  # (value, combination)
    for j, col in enumerate(columns):
        v, c = col, 1 << j
        for rv, rc in rows:
            if v & (rv & -rv):
                v ^= rv
                c ^= rc
        if v:
            rows.append((v, c))
    v, c = target, 0
    for rv, rc in rows:
        if v & (rv & -rv):
            v ^= rv
            c ^= rc
    if v:
        raise RuntimeError("target not in the span of the product terms")
    return c


def product_matrix(n_bits, mul, forms):
    """Matrix (list of masks over the product terms, one per output bit) of a
    field product whose terms are forms(a)[j] AND forms(b)[j]."""
    n = 1 << n_bits
    cols, targets = [], [0] * n_bits
    nterm = len(forms([1 << i for i in range(n_bits)]))
    col_vals = [0] * nterm
    idx = 0
    for a in range(n):
        for b in range(n):
            fa = forms([(a >> i) & 1 for i in range(n_bits)])
            fb = forms([(b >> i) & 1 for i in range(n_bits)])
            for j in range(nterm):
                if fa[j] & fb[j]:
                    col_vals[j] |= 1 << idx
            prod = mul(a, b)
            for r in range(n_bits):
                if (prod >> r) & 1:
                    targets[r] |= 1 << idx
            idx += 1
    return [solve_gf2(col_vals, t) for t in targets]


def build(nu=NU, lam=LAM, beta=BETA, seed=SEED):
    rng = random.Random(seed)
    M = aes_roots(nu, lam)[beta]
    Minv = mat_inverse(M)
    AMinv = [affine(mat_apply(Minv, 1 << i)) for i in range(8)]
    m16 = lambda a, b: g16_mul(a, b, nu)
    C16 = product_matrix(4, m16, forms9)
    C4 = product_matrix(2, g4_mul, forms3)
    circ = Circuit(8)

    # Stage A: tower bits of the input, as masks over the 8 input bits.
    xm = [sum(((M[i] >> r) & 1) << i for i in range(8)) for r in range(8)]
    x0m, x1m = xm[0:4], xm[4:8]
    f1, f0 = forms9(x1m), forms9(x0m)
    # linear part of D = lam x1^2 + x0^2 (GF(2)-linear in the tower bits)
    sq_lam = [g16_mul(lam, g16_mul(1 << i, 1 << i, nu), nu) for i in range(4)]
    sq = [g16_mul(1 << i, 1 << i, nu) for i in range(4)]
    lin = []
    for r in range(4):
        m = 0
        for i in range(4):
            if (sq_lam[i] >> r) & 1:
                m ^= x1m[i]
            if (sq[i] >> r) & 1:
                m ^= x0m[i]
        lin.append(m)
    top = linear_network(circ, list(range(8)), f1 + f0 + lin, rng)
    w1, w0, wlin = top[0:9], top[9:18], top[18:22]

    # Stage B: x1 * x0 and D.
    T1 = [circ.and_(w1[j], w0[j]) for j in range(9)]
    d_rows = [(1 << r) | (C16[r] << 4) for r in range(4)]
    D = linear_network(circ, wlin + T1, d_rows, rng)  # D bits l0, l1, h0, h1

    # Stage C: GF(16) inversion of D = a1 z + a0: d' = nu a1^2 + a1 a0 + a0^2
    # in GF(4), then D^-1 = d'^2 (a1 z + a1 + a0).
    a1m, a0m = [1 << 2, 1 << 3], [1 << 0, 1 << 1]  # GF(4) pairs (bit0, bit1) over D
    f3a1, f3a0 = forms3(a1m), forms3(a0m)
    g4sq = lambda v: g4_mul(v, v)
    lin4 = []
    for r in range(2):
        m = 0
        for i in range(2):
            if (g4_mul(nu, g4sq(1 << i)) >> r) & 1:
                m ^= a1m[i]
            if (g4sq(1 << i) >> r) & 1:
                m ^= a0m[i]
        lin4.append(m)
    cw = linear_network(circ, D, f3a1 + f3a0 + lin4 + forms3([a1m[0] ^ a0m[0], a1m[1] ^ a0m[1]]), rng)
    u1, u0, ulin, usum = cw[0:3], cw[3:6], cw[6:8], cw[8:11]
    T2 = [circ.and_(u1[j], u0[j]) for j in range(3)]
    dp = linear_network(circ, ulin + T2, [(1 << r) | (C4[r] << 2) for r in range(2)], rng)  # d' bits
    # q = d'^2: bits (q0, q1) = (d'0 ^ d'1, d'1); its 3 forms over d' bits
    qm = [0b11, 0b10]
    qf = linear_network(circ, dp, forms3(qm), rng)
    T3 = [circ.and_(qf[j], u1[j]) for j in range(3)] + [circ.and_(qf[j], usum[j]) for j in range(3)]
    di_rows = [C4[0] << 3, C4[1] << 3, C4[0], C4[1]]  # lo pair from the 2nd product, hi from the 1st
    di = linear_network(circ, T3, di_rows, rng)

    # Stage D: y1 = di x1, y0 = di (x1 + x0) = di x1 + di x0; output map.
    fd = linear_network(circ, di, forms9([1, 2, 4, 8]), rng)
    P = [circ.and_(fd[j], w1[j]) for j in range(9)]
    Q = [circ.and_(fd[j], w0[j]) for j in range(9)]
    # inv bits 0..3 = y0 = C16 P ^ C16 Q, bits 4..7 = y1 = C16 P (masks over P|Q)
    inv_masks = [C16[r] | (C16[r] << 9) for r in range(4)] + [C16[r] for r in range(4)]
    out_rows = []
    for r in range(8):
        m = 0
        for i in range(8):
            if (AMinv[i] >> r) & 1:
                m ^= inv_masks[i]
        out_rows.append(m)
    outs = linear_network(circ, P + Q, out_rows, rng)
    return circ, outs, (nu, lam, M)


def simulate(circ, outs, a):
    vals = [(a >> i) & 1 for i in range(8)]
    for op, x, y in circ.gates:
        vals.append(vals[x] ^ vals[y] if op == "^" else vals[x] & vals[y])
    return sum(vals[o] << r for r, o in enumerate(outs))


def check(circ, outs):
    for a in range(256):
        got = simulate(circ, outs, a)
        if got ^ 0x63 != sbox(a):
            raise AssertionError("circuit wrong at %d: %02x vs %02x" % (a, got ^ 0x63, sbox(a)))


def emit(circ, outs, params, path):
    n_and = sum(1 for g in circ.gates if g[0] == "&")
    n_xor = len(circ.gates) - n_and
    nu, lam, M = params
    lines = []
    lines.append("// bitsliced_sbox.cuh -- GENERATED by gen_bitsliced_sbox.py; do not edit.")
    lines.append("//")
    lines.append("// The AES S-box without its constant 0x63 (FIPS-197 sec. 5.1.1: affine map of")
    lines.append("// the inverse in GF(2^8)) as %d gates (%d AND, %d XOR), computed through the" % (len(circ.gates), n_and, n_xor))
    lines.append("// tower field GF(((2^2)^2)^2) with nu = %d, lambda = %d (tower bit patterns)." % (nu, lam))
    lines.append("// Each argument is one bit of the byte (b0 = least significant) for 32")
    lines.append("// independent bytes, one per bit of the word; the outputs overwrite the")
    lines.append("// inputs.  Checked on all 256 inputs by the generator.")
    lines.append("#pragma once")
    lines.append("#include <cstdint>")
    lines.append("#include <cuda_runtime.h>")
    lines.append("")
    lines.append("namespace gcmgpu {")
    lines.append("")
    lines.append("__host__ __device__ __forceinline__ void sbox_bitsliced(uint32_t &b0, uint32_t &b1, uint32_t &b2,")
    lines.append("                                                        uint32_t &b3, uint32_t &b4, uint32_t &b5,")
    lines.append("                                                        uint32_t &b6, uint32_t &b7)")
    lines.append("{")
    names = ["b%d" % i for i in range(8)]

    def nm(w):
        return names[w] if w < 8 else "t%d" % (w - 8)

    for gi, (op, a, b) in enumerate(circ.gates):
        lines.append("    const uint32_t t%d = %s %s %s;" % (gi, nm(a), op, nm(b)))
    for r, o in enumerate(outs):
        lines.append("    b%d = %s;" % (r, nm(o)) if o >= 8 else "    b%d = %s_in;" % (r, nm(o)))
    lines.append("}")
    lines.append("")
    lines.append("}  // namespace gcmgpu")
    # outputs that are plain inputs would need the input saved first
    if any(o < 8 for o in outs):
        raise RuntimeError("an output equals an input wire; not supported by the emitter")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")
    return len(circ.gates), n_and, n_xor


def search():
    best = None
    for nu in range(1, 4):
        for lam in range(1, 16):
            if not valid_params(nu, lam):
                continue
            for beta in aes_roots(nu, lam):
                for seed in range(8):
                    circ, outs, _ = build(nu, lam, beta, seed)
                    check(circ, outs)
                    if best is None or len(circ.gates) < best[0]:
                        best = (len(circ.gates), nu, lam, beta, seed)
                        print("gates %d: nu=%d lambda=%d beta=%d seed=%d" % best, flush=True)
    return best


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("out", nargs="?", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                           "bitsliced_sbox.cuh"))
    ap.add_argument("--search", action="store_true", help="search the parameters for the smallest circuit")
    args = ap.parse_args()
    if args.search:
        search()
        return
    circ, outs, params = build()
    check(circ, outs)
    n, na, nx = emit(circ, outs, params, args.out)
    print("wrote %s: %d gates (%d AND, %d XOR)" % (args.out, n, na, nx))


if __name__ == "__main__":
    main()
