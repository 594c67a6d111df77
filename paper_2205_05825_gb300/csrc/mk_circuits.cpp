// mk_circuits.cpp -- k-bit two's-complement operators (Sec. 3.3 and
// Sec. 4.3-4.5 of arXiv 2205.05825, Algorithms 3-6) as netlists of the
// bootstrapped gates, and their levelised evaluation on the GPU.
//
// Netlist definition (wire numbering and construction order are part of it):
//   wire 0 = constant 0, wire 1 = constant 1 (trivial ciphertexts),
//   wires 2 .. 2+ka-1 = bits of a (LSB first), then the kb bits of b,
//   gate g writes wire 2 + ka + kb + g; every gate input may be negated
//   (MKNOT, Eq. 8, is linear and folds into the next gate's linear part);
//   outputs are (wire, negated) pairs.
// Constructions:
//   full adder: t = x XOR y; s = t XOR c; cout = (x AND y) OR (t AND c)
//     (5 gates per bit; Table 3 counts 5k for the k-bit adder, Alg. 3),
//   adder: carry-in 0, last carry computed and dropped;
//   subtractor (Alg. 5): a + NOT(b) + 1 (carry-in 1);
//   multiplier (Alg. 4): Baugh-Wooley partial products (NAND for the
//     mixed-sign terms, constant ones at columns k and 2k-1), column
//     compression with full adders, a final ripple addition; 2k-bit product;
//   divider (Alg. 6): compensation devices to magnitudes, a non-restoring
//     array of CAS cells (Sec. 4.5: out = a XOR ((b XOR p) XOR c),
//     cout = ((a OR c) AND (b XOR p)) OR (a AND c)), a remainder correction,
//     compensation back; quotient sign = sign(a) XOR sign(b), remainder with
//     a's sign (truncating division).
// Those are the array family (MK_CIRCUIT_ARRAY): ripple carry chains, O(k)
// levels per addition, the fewest gates.  The shallow family
// (MK_CIRCUIT_SHALLOW) computes the same functions with every carry chain
// replaced by a Sklansky parallel-prefix carry network (generate x AND y,
// propagate x XOR y, the associative combine (G, P) o (G', P') =
// (G OR (P AND G'), P AND P') over the carry-in and the bits, sums
// p XOR carry): the adder and subtractor, every row of the non-restoring
// divider (operand b XOR p, carry-in p), its remainder correction and every
// compensation increment; the multiplier reduces its Baugh-Wooley partial
// products by Dadda stages (targets 2, 3, 4, 6, 9, ...) and adds the two
// remaining rows with the prefix adder.  Gates with a constant input are
// folded away and gates nobody reads are pruned.  O(log k) levels per
// addition (the 16-bit divider: 852 -> 223 levels) for 10-25 % more gates
// in the multiplier and divider and up to 60 % more in the adders: a level
// is one batched launch whatever its width, so depth is what a narrow,
// latency-bound evaluation pays for.
// Two more families for comparison with the paper's own constructions:
// MK_CIRCUIT_PAPER keeps the array family's adder, subtractor and divider and
// builds the multiplier from the paper's 0-, 1- and 2-adders (Sec. 3.3,
// Alg. 4; Fig. 1 is missing, this is a reading of its rules): each signal
// carries the sign of its weight -- a partial product a_j b_i weighs
// -2^(i+j) when exactly one of i, j is k - 1 -- and a full adder whose inputs
// include t of negative weight negates them first (NOT is free) and then
// outputs, for t = 0, 1, 2, 3: sum +, carry +; NOT(sum) -, carry + (the
// 1-adder); sum +, NOT(carry) - (the 2-adder); sum -, carry -.  The k^2
// partial products come first (row i, then column j); rows i = 1 .. k-1
// have k-1 adders each (column j adds row i's partial product of column j
// to the running sum and carry of weight i + j; the first row's carries are
// the constant 0) and pass row i's last partial product through; a last
// row of k-1 adders ripples the sums and carries of weights k .. 2k-2 from
// a carry-in of 0 taken as negative, so that each of its adders is a
// 2-adder and its final carry, of negative weight, is the sign bit of the
// 2k-bit product: k rows of k-1 adders, k^2 + 5 k (k-1) gates.
// MK_CIRCUIT_NAND is the naive scheme of Table 2: the array family with
// every gate composed of bootstrapped NAND gates only, the one gate of the
// scheme the paper starts from; a negated input or output costs NAND(x, x)
// (a negated constant is the other constant); AND = NAND(n, n),
// n = NAND(x, y); OR = NAND(NAND(x, x), NAND(y, y)); NOR = NAND(o, o) of that
// OR; XOR = NAND(NAND(x, n), NAND(y, n)), n = NAND(x, y); XNOR = NAND(x', x')
// of that XOR.
// Levels: a gate's level is 1 + the deepest of its inputs; each level is one
// batched bootstrap + key-switch launch over all its gates of all pairs.
#include <algorithm>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "mk_internal.h"

namespace mk {


namespace {

enum { OP_AND = MK_AND, OP_OR = MK_OR, OP_NAND = MK_NAND, OP_NOR = MK_NOR, OP_XOR = MK_XOR, OP_XNOR = MK_XNOR };

const Wire kZero{0, 0}, kOne{1, 0};

Wire negw(Wire x) { return Wire{x.w, 1 - x.neg}; }

struct Builder {
    Netlist net;
    std::vector<Wire> A, B;
    Builder(uint32_t ka, uint32_t kb) {
        net.ka = ka;
        net.kb = kb;
        for (uint32_t i = 0; i < ka; ++i) A.push_back(Wire{(int32_t)(2 + i), 0});
        for (uint32_t i = 0; i < kb; ++i) B.push_back(Wire{(int32_t)(2 + ka + i), 0});
    }
    Wire gate(int op, Wire x, Wire y) {
        mk_gate_rec r{};
        r.op = (uint8_t)op;
        r.neg_a = (uint8_t)x.neg;
        r.neg_b = (uint8_t)y.neg;
        r.a = x.w;
        r.b = y.w;
        net.gates.push_back(r);
        return Wire{(int32_t)(2 + net.ka + net.kb + net.gates.size() - 1), 0};
    }
    std::pair<Wire, Wire> full_adder(Wire x, Wire y, Wire c) {
        Wire t = gate(OP_XOR, x, y);
        Wire s = gate(OP_XOR, t, c);
        Wire g1 = gate(OP_AND, x, y);
        Wire g2 = gate(OP_AND, t, c);
        return {s, gate(OP_OR, g1, g2)};
    }
    std::pair<Wire, Wire> half_adder(Wire x, Wire y) {
        Wire s = gate(OP_XOR, x, y);
        return {s, gate(OP_AND, x, y)};
    }
    std::vector<Wire> compensate(const std::vector<Wire> &bits, Wire sign) {
        std::vector<Wire> out;
        Wire c = sign;
        for (const Wire &x : bits) {
            Wire t = gate(OP_XOR, x, sign);
            out.push_back(gate(OP_XOR, t, c));
            c = gate(OP_AND, t, c);
        }
        return out;
    }
};

// ---------------------------------------------------------------- shallow family
// Value of a constant wire reference (0 or 1), else -1.
int const_value(Wire x) { return x.w <= 1 ? (x.w ^ x.neg) : -1; }

struct ShallowBuilder : Builder {
    using Builder::Builder;
    Wire and_(Wire x, Wire y) {
        const int cx = const_value(x), cy = const_value(y);
        if (cx == 0 || cy == 0) return kZero;
        if (cx == 1) return y;
        if (cy == 1) return x;
        return gate(OP_AND, x, y);
    }
    Wire or_(Wire x, Wire y) {
        const int cx = const_value(x), cy = const_value(y);
        if (cx == 1 || cy == 1) return kOne;
        if (cx == 0) return y;
        if (cy == 0) return x;
        return gate(OP_OR, x, y);
    }
    Wire xor_(Wire x, Wire y) {
        const int cx = const_value(x), cy = const_value(y);
        if (cx >= 0 && cy >= 0) return (cx ^ cy) ? kOne : kZero;
        if (cx >= 0) return cx ? negw(y) : y;
        if (cy >= 0) return cy ? negw(x) : x;
        return gate(OP_XOR, x, y);
    }
    // Sum bits of xs + ys + cin (xs.size() bits, carry out dropped).  Element
    // 0 is (cin, 0), element i >= 1 is (g, p) of bit i - 1; the Sklansky
    // network leaves in element i the group (G, P) of elements 0..i, whose G
    // is the carry into bit i.
    std::vector<Wire> prefix_add(const std::vector<Wire> &xs, const std::vector<Wire> &ys, Wire cin) {
        const size_t n = xs.size();
        std::vector<Wire> g, p;
        for (size_t i = 0; i < n; ++i) {
            g.push_back(and_(xs[i], ys[i]));
            p.push_back(xor_(xs[i], ys[i]));
        }
        std::vector<Wire> G{cin}, P{kZero};
        for (size_t i = 0; i + 1 < n; ++i) {
            G.push_back(g[i]);
            P.push_back(p[i]);
        }
        for (size_t d = 0; ((size_t)1 << d) < n; ++d)
            for (size_t i = 0; i < n; ++i)
                if ((i >> d) & 1) {
                    const size_t j = ((i >> d) << d) - 1;  // top element of the lower half-block
                    const Wire t = and_(P[i], G[j]);
                    G[i] = or_(G[i], t);
                    P[i] = and_(P[i], P[j]);
                }
        std::vector<Wire> sum;
        for (size_t i = 0; i < n; ++i) sum.push_back(xor_(p[i], G[i]));
        return sum;
    }
    // Conditional two's complement: (bits XOR sign) + sign.
    std::vector<Wire> compensate_prefix(const std::vector<Wire> &bits, Wire sign) {
        std::vector<Wire> t;
        for (const Wire &x : bits) t.push_back(xor_(x, sign));
        return prefix_add(t, std::vector<Wire>(t.size(), kZero), sign);
    }
};

// Drop gates whose outputs no output depends on; renumber the rest in
// construction order.
Netlist prune(const Netlist &net) {
    const int32_t base = (int32_t)(2 + net.ka + net.kb);
    std::vector<char> live(base + net.gates.size(), 0);
    for (const Wire &o : net.outputs) live[o.w] = 1;
    for (size_t g = net.gates.size(); g-- > 0;)
        if (live[base + g]) live[net.gates[g].a] = live[net.gates[g].b] = 1;
    std::vector<int32_t> id(base + net.gates.size());
    for (int32_t w = 0; w < base; ++w) id[w] = w;
    Netlist out;
    out.ka = net.ka;
    out.kb = net.kb;
    for (size_t g = 0; g < net.gates.size(); ++g) {
        if (!live[base + g]) continue;
        mk_gate_rec r = net.gates[g];
        r.a = id[r.a];
        r.b = id[r.b];
        id[base + g] = base + (int32_t)out.gates.size();
        out.gates.push_back(r);
    }
    for (const Wire &o : net.outputs) out.outputs.push_back(Wire{id[o.w], o.neg});
    return out;
}

Netlist build_shallow_adder(uint32_t k, bool subtract) {
    ShallowBuilder b(k, k);
    std::vector<Wire> ys;
    for (uint32_t i = 0; i < k; ++i) ys.push_back(subtract ? negw(b.B[i]) : b.B[i]);
    b.net.outputs = b.prefix_add(b.A, ys, subtract ? kOne : kZero);
    return prune(b.net);
}

Netlist build_shallow_multiplier(uint32_t k) {
    ShallowBuilder b(k, k);
    std::vector<std::vector<Wire>> cols(2 * k);
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j) {
            const int op = ((i == k - 1) != (j == k - 1)) ? OP_NAND : OP_AND;
            cols[i + j].push_back(b.gate(op, b.A[j], b.B[i]));
        }
    cols[k].push_back(kOne);
    cols[2 * k - 1].push_back(kOne);
    // Dadda stages: targets 2, 3, 4, 6, 9, ... below the tallest column
    size_t tallest = 0;
    for (const auto &c : cols) tallest = std::max(tallest, c.size());
    std::vector<size_t> targets{2};
    while (targets.back() < tallest) targets.push_back(targets.back() * 3 / 2);
    for (size_t t = targets.size() - 1; t-- > 0;) {
        const size_t d = targets[t];
        std::vector<std::vector<Wire>> nw(2 * k), carries(2 * k + 1);
        for (uint32_t c = 0; c < 2 * k; ++c) {
            std::vector<Wire> bits = cols[c];
            size_t pos = 0, h = bits.size() + carries[c].size();
            while (h > d) {
                std::pair<Wire, Wire> sc;
                if (h - d >= 2) {
                    sc = b.full_adder(bits[pos], bits[pos + 1], bits[pos + 2]);
                    pos += 3;
                    h -= 2;
                } else {
                    sc = b.half_adder(bits[pos], bits[pos + 1]);
                    pos += 2;
                    h -= 1;
                }
                nw[c].push_back(sc.first);
                carries[c + 1].push_back(sc.second);
            }
            for (; pos < bits.size(); ++pos) nw[c].push_back(bits[pos]);
            for (const Wire &w : carries[c]) nw[c].push_back(w);
        }
        cols.swap(nw);
    }
    std::vector<Wire> xs, ys;
    for (uint32_t c = 0; c < 2 * k; ++c) {
        xs.push_back(cols[c].size() >= 1 ? cols[c][0] : kZero);
        ys.push_back(cols[c].size() >= 2 ? cols[c][1] : kZero);
    }
    b.net.outputs = b.prefix_add(xs, ys, kZero);
    return prune(b.net);
}

Netlist build_shallow_divider(uint32_t k) {
    ShallowBuilder b(k, k);
    const Wire sa = b.A[k - 1], sb = b.B[k - 1];
    std::vector<Wire> A = b.compensate_prefix(b.A, sa);
    std::vector<Wire> D = b.compensate_prefix(b.B, sb);
    D.push_back(kZero);
    std::vector<Wire> R(k + 1, kZero);
    Wire p = kOne;
    std::vector<Wire> q(k);
    for (int i = (int)k - 1; i >= 0; --i) {
        std::vector<Wire> sh{A[i]};
        for (uint32_t j = 0; j < k; ++j) sh.push_back(R[j]);
        std::vector<Wire> ys;
        for (uint32_t j = 0; j <= k; ++j) ys.push_back(b.xor_(D[j], p));
        R = b.prefix_add(sh, ys, p);  // R + (p ? -D : D)
        q[i] = negw(R[k]);
        p = q[i];
    }
    const Wire s = R[k];
    std::vector<Wire> m, low(R.begin(), R.begin() + k);
    for (uint32_t j = 0; j < k; ++j) m.push_back(b.and_(D[j], s));
    std::vector<Wire> rmag = b.prefix_add(low, m, kZero);
    const Wire qs = b.xor_(sa, sb);
    std::vector<Wire> qo = b.compensate_prefix(q, qs);
    std::vector<Wire> ro = b.compensate_prefix(rmag, sa);
    b.net.outputs = qo;
    b.net.outputs.insert(b.net.outputs.end(), ro.begin(), ro.end());
    return prune(b.net);
}

Netlist build_adder(uint32_t k, bool subtract) {
    Builder b(k, k);
    Wire c = subtract ? kOne : kZero;
    for (uint32_t i = 0; i < k; ++i) {
        Wire y = subtract ? negw(b.B[i]) : b.B[i];
        auto sc = b.full_adder(b.A[i], y, c);
        b.net.outputs.push_back(sc.first);
        c = sc.second;
    }
    return b.net;
}

Netlist build_multiplier(uint32_t k) {
    Builder b(k, k);
    std::vector<std::vector<Wire>> cols(2 * k);
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j) {
            const int op = ((i == k - 1) != (j == k - 1)) ? OP_NAND : OP_AND;
            cols[i + j].push_back(b.gate(op, b.A[j], b.B[i]));
        }
    cols[k].push_back(kOne);
    cols[2 * k - 1].push_back(kOne);
    auto tall = [&]() {
        for (auto &c : cols)
            if (c.size() > 2) return true;
        return false;
    };
    while (tall()) {
        std::vector<std::vector<Wire>> nw(2 * k);
        for (uint32_t c = 0; c < 2 * k; ++c) {
            size_t pos = 0;
            const std::vector<Wire> &bits = cols[c];
            while (bits.size() - pos >= 3) {
                auto sc = b.full_adder(bits[pos], bits[pos + 1], bits[pos + 2]);
                pos += 3;
                nw[c].push_back(sc.first);
                if (c + 1 < 2 * k) nw[c + 1].push_back(sc.second);
            }
            for (; pos < bits.size(); ++pos) nw[c].push_back(bits[pos]);
        }
        cols.swap(nw);
    }
    bool have_carry = false;
    Wire carry{};
    for (uint32_t c = 0; c < 2 * k; ++c) {
        std::vector<Wire> bits = cols[c];
        if (have_carry) bits.push_back(carry);
        if (bits.size() == 3) {
            auto sc = b.full_adder(bits[0], bits[1], bits[2]);
            b.net.outputs.push_back(sc.first);
            carry = sc.second;
            have_carry = true;
        } else if (bits.size() == 2) {
            auto sc = b.half_adder(bits[0], bits[1]);
            b.net.outputs.push_back(sc.first);
            carry = sc.second;
            have_carry = true;
        } else if (bits.size() == 1) {
            b.net.outputs.push_back(bits[0]);
            have_carry = false;
        } else {
            b.net.outputs.push_back(kZero);
            have_carry = false;
        }
    }
    return b.net;
}

Netlist build_divider(uint32_t k) {
    Builder b(k, k);
    const Wire sa = b.A[k - 1], sb = b.B[k - 1];
    std::vector<Wire> A = b.compensate(b.A, sa);
    std::vector<Wire> D = b.compensate(b.B, sb);
    D.push_back(kZero);
    std::vector<Wire> R(k + 1, kZero);
    Wire p = kOne;
    std::vector<Wire> q(k);
    for (int i = (int)k - 1; i >= 0; --i) {
        std::vector<Wire> sh;
        sh.push_back(A[i]);
        for (uint32_t j = 0; j < k; ++j) sh.push_back(R[j]);
        R.swap(sh);
        Wire c = p;
        std::vector<Wire> nr;
        for (uint32_t j = 0; j <= k; ++j) {
            Wire bp = b.gate(OP_XOR, D[j], p);
            Wire inner = b.gate(OP_XOR, bp, c);
            nr.push_back(b.gate(OP_XOR, R[j], inner));
            Wire aoc = b.gate(OP_OR, R[j], c);
            Wire t = b.gate(OP_AND, aoc, bp);
            Wire ac = b.gate(OP_AND, R[j], c);
            c = b.gate(OP_OR, t, ac);
        }
        R.swap(nr);
        q[i] = negw(R[k]);
        p = q[i];
    }
    const Wire s = R[k];
    Wire c = kZero;
    std::vector<Wire> rmag;
    for (uint32_t j = 0; j < k; ++j) {
        Wire m = b.gate(OP_AND, D[j], s);
        auto sc = b.full_adder(R[j], m, c);
        rmag.push_back(sc.first);
        c = sc.second;
    }
    const Wire qs = b.gate(OP_XOR, sa, sb);
    std::vector<Wire> qo = b.compensate(q, qs);
    std::vector<Wire> ro = b.compensate(rmag, sa);
    b.net.outputs = qo;
    b.net.outputs.insert(b.net.outputs.end(), ro.begin(), ro.end());
    return b.net;
}

// ---------------------------------------------------------------- the paper's multiplier
// A signal and the sign of its weight (1: it counts -2^w).
struct Signed {
    Wire r;
    int negw;
};

// Full adder of three signals of one weight, typed by how many weigh
// negative: the sum at that weight and the carry at the next, with their signs.
std::pair<Signed, Signed> typed_adder(Builder &b, const Signed &x, const Signed &y, const Signed &z) {
    const int t = x.negw + y.negw + z.negw;
    const bool flip = t == 1 || t == 2;
    const Wire ix = (flip && x.negw) ? negw(x.r) : x.r;
    const Wire iy = (flip && y.negw) ? negw(y.r) : y.r;
    const Wire iz = (flip && z.negw) ? negw(z.r) : z.r;
    const std::pair<Wire, Wire> sc = b.full_adder(ix, iy, iz);
    switch (t) {
    case 0: return {Signed{sc.first, 0}, Signed{sc.second, 0}};
    case 1: return {Signed{negw(sc.first), 1}, Signed{sc.second, 0}};
    case 2: return {Signed{sc.first, 0}, Signed{negw(sc.second), 1}};
    default: return {Signed{sc.first, 1}, Signed{sc.second, 1}};
    }
}

bool build_paper_multiplier(uint32_t k, Netlist &out) {
    Builder b(k, k);
    std::vector<std::vector<Signed>> pp(k, std::vector<Signed>(k));
    for (uint32_t i = 0; i < k; ++i)
        for (uint32_t j = 0; j < k; ++j)
            pp[i][j] = Signed{b.gate(OP_AND, b.A[j], b.B[i]), ((i == k - 1) != (j == k - 1)) ? 1 : 0};
    const Signed zero{kZero, 0};
    std::vector<Signed> S(2 * k, zero), C(2 * k, zero), res;
    for (uint32_t w = 0; w < k; ++w) S[w] = pp[0][w];
    res.push_back(pp[0][0]);
    for (uint32_t i = 1; i < k; ++i) {
        std::vector<Signed> S2(2 * k, zero), C2(2 * k, zero);
        for (uint32_t j = 0; j + 1 < k; ++j) {
            const uint32_t w = i + j;
            const std::pair<Signed, Signed> sc = typed_adder(b, pp[i][j], S[w], C[w]);
            S2[w] = sc.first;
            C2[w + 1] = sc.second;
        }
        S2[i + k - 1] = pp[i][k - 1];
        S = S2;
        C = C2;
        res.push_back(S[i]);
    }
    Signed carry{kZero, 1};  // a zero of negative weight: every adder of the last row is a 2-adder
    for (uint32_t w = k; w + 1 < 2 * k; ++w) {
        const std::pair<Signed, Signed> sc = typed_adder(b, S[w], C[w], carry);
        res.push_back(sc.first);
        carry = sc.second;
    }
    res.push_back(carry);
    for (size_t w = 0; w < res.size(); ++w)  // two's complement: only the top bit weighs negative
        if (res[w].negw != (w + 1 == res.size() ? 1 : 0)) return false;
    for (const Signed &x : res) b.net.outputs.push_back(x.r);
    out = b.net;
    return true;
}

// ---------------------------------------------------------------- the naive NAND-only scheme
Netlist nand_only(const Netlist &net) {
    Builder b(net.ka, net.kb);
    const int32_t base = (int32_t)(2 + net.ka + net.kb);
    std::vector<Wire> new_of(net.gates.size());
    auto plain = [&](int32_t w, int ng) -> Wire {
        const Wire r = w >= base ? new_of[(size_t)(w - base)] : Wire{w, 0};
        if (!ng) return r;
        if (r.w <= 1) return Wire{1 - r.w, 0};  // a constant: negated for free
        return b.gate(OP_NAND, r, r);
    };
    for (size_t g = 0; g < net.gates.size(); ++g) {
        const mk_gate_rec &G = net.gates[g];
        const Wire x = plain(G.a, G.neg_a);
        const Wire y = plain(G.b, G.neg_b);
        Wire r;
        if (G.op == OP_NAND) {
            r = b.gate(OP_NAND, x, y);
        } else if (G.op == OP_AND) {
            const Wire n = b.gate(OP_NAND, x, y);
            r = b.gate(OP_NAND, n, n);
        } else if (G.op == OP_OR || G.op == OP_NOR) {
            const Wire nx = b.gate(OP_NAND, x, x);
            const Wire ny = b.gate(OP_NAND, y, y);
            r = b.gate(OP_NAND, nx, ny);
            if (G.op == OP_NOR) r = b.gate(OP_NAND, r, r);
        } else {  // XOR, XNOR
            const Wire n = b.gate(OP_NAND, x, y);
            const Wire p = b.gate(OP_NAND, x, n);
            const Wire q = b.gate(OP_NAND, y, n);
            r = b.gate(OP_NAND, p, q);
            if (G.op == OP_XNOR) r = b.gate(OP_NAND, r, r);
        }
        new_of[g] = r;
    }
    for (const Wire &o : net.outputs) b.net.outputs.push_back(plain(o.w, o.neg));
    return b.net;
}

}  // namespace

bool build_netlist(int op, uint32_t k, int style, Netlist &out) {
    if (k < 2 || k > 64) return false;
    if (style == MK_CIRCUIT_NAND) {
        Netlist array;
        if (!build_netlist(op, k, MK_CIRCUIT_ARRAY, array)) return false;
        out = nand_only(array);
        return true;
    }
    if (style == MK_CIRCUIT_PAPER) {
        if (op == MK_OP_MUL) return build_paper_multiplier(k, out);
        return build_netlist(op, k, MK_CIRCUIT_ARRAY, out);
    }
    if (style == MK_CIRCUIT_SHALLOW) {
        switch (op) {
        case MK_OP_ADD: out = build_shallow_adder(k, false); return true;
        case MK_OP_SUB: out = build_shallow_adder(k, true); return true;
        case MK_OP_MUL: out = build_shallow_multiplier(k); return true;
        case MK_OP_DIV: out = build_shallow_divider(k); return true;
        default: return false;
        }
    }
    if (style != MK_CIRCUIT_ARRAY) return false;
    switch (op) {
    case MK_OP_ADD: out = build_adder(k, false); return true;
    case MK_OP_SUB: out = build_adder(k, true); return true;
    case MK_OP_MUL: out = build_multiplier(k); return true;
    case MK_OP_DIV: out = build_divider(k); return true;
    default: return false;
    }
}

// (cst, s1, s2) of a gate with possibly negated inputs: NOT(c) = 1/4 - c, so
// s * NOT(c) = s/4 - s*c.
mk_lin gate_lin(const mk_gate_rec &g) {
    static const uint32_t cst[6] = {0xE0000000u, 0x20000000u, 0xA0000000u, 0x60000000u, 0x0u, 0x80000000u};
    static const int32_t s1[6] = {1, 1, -1, -1, 2, 2};
    static const int32_t s2[6] = {1, 1, -1, -1, -2, -2};
    mk_lin L{cst[g.op], s1[g.op], s2[g.op]};
    if (g.neg_a) {
        L.cst += (uint32_t)L.s1 << 30;
        L.s1 = -L.s1;
    }
    if (g.neg_b) {
        L.cst += (uint32_t)L.s2 << 30;
        L.s2 = -L.s2;
    }
    return L;
}

std::vector<uint32_t> netlist_levels(const Netlist &net) {
    const uint32_t base = 2 + net.ka + net.kb;
    std::vector<uint32_t> lev(base + net.gates.size(), 0), out(net.gates.size());
    for (size_t g = 0; g < net.gates.size(); ++g) {
        const uint32_t L = 1 + std::max(lev[net.gates[g].a], lev[net.gates[g].b]);
        lev[base + g] = L;
        out[g] = L;
    }
    return out;
}

}  // namespace mk

extern "C" int mk_gate_lin(int type, int neg_a, int neg_b, mk_lin *out) {
    if (type < 0 || type > 5 || !out) return MK_EINVAL;
    mk_gate_rec g{};
    g.op = (uint8_t)type;
    g.neg_a = neg_a ? 1 : 0;
    g.neg_b = neg_b ? 1 : 0;
    *out = mk::gate_lin(g);
    return MK_OK;
}
