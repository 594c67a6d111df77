"""Netlists of the k-bit two's-complement operators (test infrastructure only).

Written from the paper's descriptions (Sec. 3.3, Sec. 4.3-4.5, Algorithms 3-6)
under these readings:
  - full adder (Sec. 3.3, Alg. 3): t = a XOR b; s = t XOR c;
    cout = (a AND b) OR (t AND c) -- 5 bootstrapped gates per bit, carry-in
    0, the last carry computed and dropped, so 5k gates as in Table 3;
  - subtractor (Alg. 5): a + NOT(b) + 1, NOT folded into the next gate's
    linear part (MKNOT is linear, Eq. 8);
  - multiplier (Alg. 4, two's complement): Baugh-Wooley partial products
    (NAND for the mixed-sign terms, constants 1 at columns k and 2k-1),
    column compression with full adders, final ripple addition; the 2k-bit
    product;
  - divider (Alg. 6): compensation devices (XOR with the sign, then add the
    sign) to magnitudes, a non-restoring array of CAS cells
    (out = a XOR ((b XOR p) XOR c), cout = ((a OR c) AND (b XOR p)) OR (a AND c)),
    a final remainder correction, and compensation back to two's complement;
    quotient sign = sign(a) XOR sign(b), remainder takes a's sign.

Four construction families ("styles") compute the same functions:
  - "array": the constructions above, with their ripple carry chains (O(k)
    levels per addition; the fewest gates);
  - "shallow": every carry chain replaced by a Sklansky parallel-prefix
    carry network (generate g = x AND y, propagate p = x XOR y, the
    associative combine (G, P) o (G', P') = (G OR (P AND G'), P AND P') over
    the carry-in and the bits, sums p XOR carry): the adder and subtractor,
    the multiplier's final addition, every row of the non-restoring divider
    (row operand b XOR p, carry-in p) and every compensation increment.
    The partial products, the column compression and the divider's row
    recurrence are those of the array family.  Gates with a constant input
    are folded away (AND with 0 is 0, XOR with 1 is a negated wire, ...) and
    gates whose outputs are never read are pruned.  O(log k) levels per
    addition, for 10-25 % more gates in the multiplier and divider and up to
    60 % more in the adders;
  - "paper": the array family's adder, subtractor and divider, and the
    multiplier of Sec. 3.3 / Alg. 4 built from the paper's 0-, 1- and
    2-adders (reading of the missing Fig. 1): every signal carries the sign
    of its weight (a partial product a_j b_i weighs -2^(i+j) when exactly
    one of i, j is k - 1); a full adder with t inputs of negative weight
    first negates those inputs (NOT is free) and then: t = 0 both outputs
    positive; t = 1 (the 1-adder) the sum is negated and weighs negative,
    the carry positive; t = 2 (the 2-adder) the sum positive, the carry
    negated and negative; t = 3 neither is negated, both negative.  The
    k^2 partial products come first (row i, then column j); rows i = 1 ..
    k - 1 each have k - 1 adders (column j adds the partial product of row
    i, column j, to the running sum and carry at weight i + j; the first
    row's carries are the constant 0), the last partial product of each row
    passes through, and a final row of k - 1 adders ripples the sums and
    carries of weights k .. 2k - 2 with a carry-in of 0 taken as negative,
    so that every adder of that row is a 2-adder; its last carry, of
    negative weight, is the sign bit of the 2k-bit product.  k rows of
    k - 1 adders, k^2 + 5 k (k - 1) gates;
  - "nand": the naive scheme of Table 2: the array family's netlists with
    every gate composed of bootstrapped NAND gates only (the one gate the
    underlying scheme provides): a negated input or output costs NAND(x, x)
    (constants are negated for free); AND = NAND(n, n) with n = NAND(x, y);
    OR = NAND(NAND(x, x), NAND(y, y)); NOR = NAND(o, o) with o that OR;
    XOR = NAND(NAND(x, n), NAND(y, n)) with n = NAND(x, y); XNOR =
    NAND(x', x') with x' that XOR.

A netlist is a dict: ka, kb (input widths), gates = list of
(op, a, neg_a, b, neg_b) with op in 0..5 (AND, OR, NAND, NOR, XOR, XNOR) and
output wire 2 + ka + kb + index; wires 0 and 1 are the constants 0 and 1,
wires 2..2+ka-1 the bits of a (LSB first), then the bits of b; outputs =
list of (wire, negated).  The construction order below is part of the
definition (the library builds the identical netlist).
"""
AND, OR, NAND, NOR, XOR, XNOR = range(6)
OPS = {"add": 0, "sub": 1, "mul": 2, "div": 3}


class _Builder:
    def __init__(self, ka, kb):
        self.ka, self.kb = ka, kb
        self.gates = []
        self.A = [(2 + i, 0) for i in range(ka)]
        self.B = [(2 + ka + i, 0) for i in range(kb)]

    def gate(self, op, x, y):
        self.gates.append((op, x[0], x[1], y[0], y[1]))
        return (2 + self.ka + self.kb + len(self.gates) - 1, 0)

    def full_adder(self, x, y, c):
        t = self.gate(XOR, x, y)
        s = self.gate(XOR, t, c)
        g1 = self.gate(AND, x, y)
        g2 = self.gate(AND, t, c)
        return s, self.gate(OR, g1, g2)

    def half_adder(self, x, y):
        return self.gate(XOR, x, y), self.gate(AND, x, y)


ZERO, ONE = (0, 0), (1, 0)


def neg(w):
    return (w[0], 1 - w[1])


def adder(k, subtract=False):
    bld = _Builder(k, k)
    c = ONE if subtract else ZERO
    out = []
    for i in range(k):
        y = neg(bld.B[i]) if subtract else bld.B[i]
        s, c = bld.full_adder(bld.A[i], y, c)
        out.append(s)
    return dict(ka=k, kb=k, gates=bld.gates, outputs=out)


def multiplier(k):
    bld = _Builder(k, k)
    cols = [[] for _ in range(2 * k)]
    for i in range(k):
        for j in range(k):
            op = NAND if (i == k - 1) != (j == k - 1) else AND
            cols[i + j].append(bld.gate(op, bld.A[j], bld.B[i]))
    cols[k].append(ONE)
    cols[2 * k - 1].append(ONE)
    while any(len(c) > 2 for c in cols):
        new = [[] for _ in range(2 * k)]
        for c in range(2 * k):
            bits = cols[c]
            while len(bits) >= 3:
                s, co = bld.full_adder(bits[0], bits[1], bits[2])
                bits = bits[3:]
                new[c].append(s)
                if c + 1 < 2 * k:
                    new[c + 1].append(co)
            new[c].extend(bits)
        cols = new
    out, carry = [], None
    for c in range(2 * k):
        bits = list(cols[c]) + ([carry] if carry is not None else [])
        if len(bits) == 3:
            s, carry = bld.full_adder(bits[0], bits[1], bits[2])
        elif len(bits) == 2:
            s, carry = bld.half_adder(bits[0], bits[1])
        elif len(bits) == 1:
            s, carry = bits[0], None
        else:
            s, carry = ZERO, None
        out.append(s)
    return dict(ka=k, kb=k, gates=bld.gates, outputs=out)


def _compensate(bld, bits, sign):
    """Conditional two's complement: XOR every bit with the sign, then add the sign."""
    out, c = [], sign
    for x in bits:
        t = bld.gate(XOR, x, sign)
        out.append(bld.gate(XOR, t, c))
        c = bld.gate(AND, t, c)
    return out


def divider(k):
    bld = _Builder(k, k)
    sa, sb = bld.A[k - 1], bld.B[k - 1]
    A = _compensate(bld, bld.A, sa)              # |a|, k bits unsigned
    D = _compensate(bld, bld.B, sb) + [ZERO]     # |b| zero-extended to k+1 bits
    R = [ZERO] * (k + 1)                         # partial remainder, k+1 bits signed
    p = ONE                                      # first row subtracts
    q = [None] * k
    for i in range(k - 1, -1, -1):
        R = [A[i]] + R[:k]                       # R = 2R + a_i (top bit shifted out)
        c = p
        new = []
        for j in range(k + 1):                   # CAS cells, LSB first
            bp = bld.gate(XOR, D[j], p)
            new.append(bld.gate(XOR, R[j], bld.gate(XOR, bp, c)))
            aoc = bld.gate(OR, R[j], c)
            t = bld.gate(AND, aoc, bp)
            ac = bld.gate(AND, R[j], c)
            c = bld.gate(OR, t, ac)
        R = new
        q[i] = neg(R[k])                         # q_i = 1 iff the new remainder is >= 0
        p = q[i]
    s = R[k]                                     # remainder negative: add |b| back
    c = ZERO
    rmag = []
    for j in range(k):
        m = bld.gate(AND, D[j], s)
        r, c = bld.full_adder(R[j], m, c)
        rmag.append(r)
    qs = bld.gate(XOR, sa, sb)
    qout = _compensate(bld, q, qs)
    rout = _compensate(bld, rmag, sa)
    return dict(ka=k, kb=k, gates=bld.gates, outputs=qout + rout)


# ----------------------------------------------------------------------------- shallow family
def _const(w):
    """Value of a constant wire reference, else None."""
    return w[0] ^ w[1] if w[0] in (0, 1) else None


class _Shallow(_Builder):
    """Builder whose AND / OR / XOR fold constant inputs."""

    def and_(self, x, y):
        cx, cy = _const(x), _const(y)
        if cx == 0 or cy == 0:
            return ZERO
        if cx == 1:
            return y
        if cy == 1:
            return x
        return self.gate(AND, x, y)

    def or_(self, x, y):
        cx, cy = _const(x), _const(y)
        if cx == 1 or cy == 1:
            return ONE
        if cx == 0:
            return y
        if cy == 0:
            return x
        return self.gate(OR, x, y)

    def xor_(self, x, y):
        cx, cy = _const(x), _const(y)
        if cx is not None and cy is not None:
            return ONE if cx ^ cy else ZERO
        if cx is not None:
            return neg(y) if cx else y
        if cy is not None:
            return neg(x) if cy else x
        return self.gate(XOR, x, y)

    def prefix_add(self, xs, ys, cin):
        """Sum bits of xs + ys + cin (len(xs) bits, the carry out dropped).
        Element 0 is (cin, 0), element i (i >= 1) is (g, p) of bit i - 1; a
        Sklansky network leaves in element i the group (G, P) of elements
        0..i, whose G is the carry into bit i."""
        n = len(xs)
        g, p = [], []
        for x, y in zip(xs, ys):
            g.append(self.and_(x, y))
            p.append(self.xor_(x, y))
        G = [cin] + g[:n - 1]
        P = [ZERO] + p[:n - 1]
        d = 0
        while (1 << d) < n:
            for i in range(n):
                if (i >> d) & 1:
                    j = ((i >> d) << d) - 1        # top element of the lower half-block
                    t = self.and_(P[i], G[j])
                    G[i] = self.or_(G[i], t)
                    P[i] = self.and_(P[i], P[j])
            d += 1
        return [self.xor_(p[i], G[i]) for i in range(n)]

    def compensate(self, bits, sign):
        """Conditional two's complement: (bits XOR sign) + sign."""
        t = [self.xor_(x, sign) for x in bits]
        return self.prefix_add(t, [ZERO] * len(t), sign)


def prune(net):
    """Drop gates whose outputs no output depends on; renumber the rest in
    construction order."""
    base = 2 + net["ka"] + net["kb"]
    live = [False] * (base + len(net["gates"]))
    for w, _ in net["outputs"]:
        live[w] = True
    for g in range(len(net["gates"]) - 1, -1, -1):
        if live[base + g]:
            _, x, _, y, _ = net["gates"][g]
            live[x] = live[y] = True
    new_id, gates = {}, []
    for g, (op, x, nx, y, ny) in enumerate(net["gates"]):
        if live[base + g]:
            new_id[base + g] = base + len(gates)
            gates.append((op, new_id.get(x, x), nx, new_id.get(y, y), ny))
    outputs = [(new_id.get(w, w), ng) for w, ng in net["outputs"]]
    return dict(ka=net["ka"], kb=net["kb"], gates=gates, outputs=outputs)


def shallow_adder(k, subtract=False):
    bld = _Shallow(k, k)
    ys = [neg(b) for b in bld.B] if subtract else list(bld.B)
    out = bld.prefix_add(bld.A, ys, ONE if subtract else ZERO)
    return prune(dict(ka=k, kb=k, gates=bld.gates, outputs=out))


def _dadda_columns(bld, k):
    """Baugh-Wooley partial products (as in the array multiplier), then Dadda
    reduction to at most two bits per column: stage targets 2, 3, 4, 6, 9,
    ... (each 3/2 of the last), every stage bringing each column, with the
    carries it receives from the column below in that stage, down to the
    target with full adders (and a half adder when one bit too many is
    left), so that every stage adds one full-adder delay."""
    cols = [[] for _ in range(2 * k)]
    for i in range(k):
        for j in range(k):
            op = NAND if (i == k - 1) != (j == k - 1) else AND
            cols[i + j].append(bld.gate(op, bld.A[j], bld.B[i]))
    cols[k].append(ONE)
    cols[2 * k - 1].append(ONE)
    targets = [2]
    while targets[-1] < max(len(c) for c in cols):
        targets.append(targets[-1] * 3 // 2)
    for d in reversed(targets[:-1]):
        new = [[] for _ in range(2 * k)]
        carries = [[] for _ in range(2 * k + 1)]
        for c in range(2 * k):
            bits = list(cols[c])
            h = len(bits) + len(carries[c])
            while h > d:
                if h - d >= 2:
                    s, co = bld.full_adder(bits[0], bits[1], bits[2])
                    bits = bits[3:]
                    h -= 2
                else:
                    s, co = bld.half_adder(bits[0], bits[1])
                    bits = bits[2:]
                    h -= 1
                new[c].append(s)
                carries[c + 1].append(co)
            new[c].extend(bits)
            new[c].extend(carries[c])
        cols = new
    return cols


def shallow_multiplier(k):
    bld = _Shallow(k, k)
    cols = _dadda_columns(bld, k)
    xs = [c[0] if len(c) >= 1 else ZERO for c in cols]
    ys = [c[1] if len(c) >= 2 else ZERO for c in cols]
    out = bld.prefix_add(xs, ys, ZERO)
    return prune(dict(ka=k, kb=k, gates=bld.gates, outputs=out))


def shallow_divider(k):
    bld = _Shallow(k, k)
    sa, sb = bld.A[k - 1], bld.B[k - 1]
    A = bld.compensate(bld.A, sa)
    D = bld.compensate(bld.B, sb) + [ZERO]
    R = [ZERO] * (k + 1)
    p = ONE
    q = [None] * k
    for i in range(k - 1, -1, -1):
        R = [A[i]] + R[:k]
        ys = [bld.xor_(D[j], p) for j in range(k + 1)]
        R = bld.prefix_add(R, ys, p)             # R + (p ? -D : D)
        q[i] = neg(R[k])
        p = q[i]
    s = R[k]
    m = [bld.and_(D[j], s) for j in range(k)]
    rmag = bld.prefix_add(R[:k], m, ZERO)
    qs = bld.xor_(sa, sb)
    qout = bld.compensate(q, qs)
    rout = bld.compensate(rmag, sa)
    return prune(dict(ka=k, kb=k, gates=bld.gates, outputs=qout + rout))


# ----------------------------------------------------------------------------- the paper's multiplier
def paper_multiplier(k):
    """Array multiplier of the paper's 0-, 1- and 2-adders (module docstring)."""
    bld = _Builder(k, k)
    pp = [[(bld.gate(AND, bld.A[j], bld.B[i]), int((i == k - 1) != (j == k - 1))) for j in range(k)]
          for i in range(k)]

    def typed_adder(x, y, z):
        """Signed signals (wire reference, negative weight): sum at the
        inputs' weight and carry at the next, each with its weight's sign."""
        t = x[1] + y[1] + z[1]
        ins = [neg(r) if (n and t in (1, 2)) else r for r, n in (x, y, z)]
        s, c = bld.full_adder(*ins)
        if t == 0:
            return (s, 0), (c, 0)
        if t == 1:
            return (neg(s), 1), (c, 0)
        if t == 2:
            return (s, 0), (neg(c), 1)
        return (s, 1), (c, 1)

    S = {w: pp[0][w] for w in range(k)}
    C = {}
    out = [pp[0][0]]
    for i in range(1, k):
        S2, C2 = {}, {}
        for j in range(k - 1):
            w = i + j
            S2[w], C2[w + 1] = typed_adder(pp[i][j], S[w], C.get(w, (ZERO, 0)))
        S2[i + k - 1] = pp[i][k - 1]
        S, C = S2, C2
        out.append(S[i])
    carry = (ZERO, 1)  # a zero of negative weight: every adder of the last row is a 2-adder
    for w in range(k, 2 * k - 1):
        s, carry = typed_adder(S[w], C[w], carry)
        out.append(s)
    out.append(carry)
    assert [n for _, n in out] == [0] * (2 * k - 1) + [1]  # two's complement: only the top bit weighs negative
    return dict(ka=k, kb=k, gates=bld.gates, outputs=[r for r, _ in out])


# ----------------------------------------------------------------------------- the naive NAND-only scheme
def nand_only(net):
    """The netlist with every gate composed of bootstrapped NANDs (module docstring)."""
    bld = _Builder(net["ka"], net["kb"])
    base = 2 + net["ka"] + net["kb"]
    new_of = {}  # old wire -> new plain wire reference

    def plain(w, ng):
        r = new_of.get(w, (w, 0)) if w >= base else (w, 0)
        if not ng:
            return r
        if r[0] in (0, 1):
            return (1 - r[0], 0)  # a constant: negated for free
        return bld.gate(NAND, r, r)

    for g, (op, x, nx, y, ny) in enumerate(net["gates"]):
        a, b = plain(x, nx), plain(y, ny)
        if op == NAND:
            r = bld.gate(NAND, a, b)
        elif op == AND:
            n = bld.gate(NAND, a, b)
            r = bld.gate(NAND, n, n)
        elif op in (OR, NOR):
            r = bld.gate(NAND, bld.gate(NAND, a, a), bld.gate(NAND, b, b))
            if op == NOR:
                r = bld.gate(NAND, r, r)
        else:  # XOR, XNOR
            n = bld.gate(NAND, a, b)
            r = bld.gate(NAND, bld.gate(NAND, a, n), bld.gate(NAND, b, n))
            if op == XNOR:
                r = bld.gate(NAND, r, r)
        new_of[base + g] = r
    outputs = [plain(w, ng) for w, ng in net["outputs"]]
    return dict(ka=net["ka"], kb=net["kb"], gates=bld.gates, outputs=outputs)


STYLES = {"array": 0, "shallow": 1, "paper": 2, "nand": 3}


def build(op, k, style="array"):
    style = {v: n for n, v in STYLES.items()}.get(style, style)
    if style not in STYLES:
        raise ValueError(style)
    if style == "nand":
        return nand_only(build(op, k, "array"))
    if style == "paper" and op in ("mul", 2):
        return paper_multiplier(k)
    shallow = style == "shallow"
    if op in ("add", 0):
        return shallow_adder(k) if shallow else adder(k)
    if op in ("sub", 1):
        return shallow_adder(k, subtract=True) if shallow else adder(k, subtract=True)
    if op in ("mul", 2):
        return shallow_multiplier(k) if shallow else multiplier(k)
    if op in ("div", 3):
        return shallow_divider(k) if shallow else divider(k)
    raise ValueError(op)


# ----------------------------------------------------------------------------- plaintext evaluation
_FN = {AND: lambda x, y: x & y, OR: lambda x, y: x | y, NAND: lambda x, y: 1 - (x & y),
       NOR: lambda x, y: 1 - (x | y), XOR: lambda x, y: x ^ y, XNOR: lambda x, y: 1 - (x ^ y)}


def eval_plain(net, a_bits, b_bits):
    """Evaluate on plaintext bits (numpy arrays [count][ka], [count][kb] or lists)."""
    import numpy as np
    a_bits = np.asarray(a_bits, np.int64)
    b_bits = np.asarray(b_bits, np.int64)
    cnt = a_bits.shape[0]
    w = [np.zeros(cnt, np.int64), np.ones(cnt, np.int64)]
    w += [a_bits[:, i] for i in range(net["ka"])] + [b_bits[:, i] for i in range(net["kb"])]
    for op, x, nx, y, ny in net["gates"]:
        vx = w[x] ^ nx
        vy = w[y] ^ ny
        w.append(_FN[op](vx, vy))
    return np.stack([w[o] ^ ng for o, ng in net["outputs"]], axis=1)


def levels(net):
    """Level of every gate: 1 + the deepest of its inputs (inputs and constants at 0)."""
    base = 2 + net["ka"] + net["kb"]
    lev = [0] * base
    out = []
    for op, x, nx, y, ny in net["gates"]:
        L = 1 + max(lev[x], lev[y])
        lev.append(L)
        out.append(L)
    return out


# ----------------------------------------------------------------------------- encrypted evaluation
def eval_encrypted(params, keys, net, a_cts, b_cts, nthreads=None):
    """Evaluate the netlist on ciphertexts with the oracle's gates.

    a_cts, b_cts: [pairs][ka|kb][k*n+1].  Negated inputs go through MKNOT
    (Eq. 8) explicitly, then the gate's own linear part and bootstrap; gates
    of one level run as one oracle batch.  Returns [pairs][n_outputs][k*n+1].
    """
    import numpy as np
    from . import oracle as o
    a_cts = np.asarray(a_cts, np.uint32)
    b_cts = np.asarray(b_cts, np.uint32)
    P, W = a_cts.shape[0], a_cts.shape[2]
    zero = np.zeros((P, W), np.uint32)
    one = zero.copy()
    one[:, -1] = 1 << 30
    wires = [zero, one] + [a_cts[:, i] for i in range(net["ka"])] + [b_cts[:, i] for i in range(net["kb"])]
    wires += [None] * len(net["gates"])
    base = 2 + net["ka"] + net["kb"]
    lev = levels(net)

    def operand(w, ng):
        x = wires[w]
        return np.stack([o.mk_not(params, r) for r in x]) if ng else x

    for L in range(1, max(lev) + 1 if lev else 1):
        idx = [g for g, l in enumerate(lev) if l == L]
        types, xs, ys = [], [], []
        for g in idx:
            op, x, nx, y, ny = net["gates"][g]
            types += [op] * P
            xs.append(operand(x, nx))
            ys.append(operand(y, ny))
        out = o.gates(params, keys, np.array(types, np.int32), np.concatenate(xs), np.concatenate(ys),
                      nthreads=nthreads)
        for t, g in enumerate(idx):
            wires[base + g] = out[t * P:(t + 1) * P]
    res = []
    for w, ng in net["outputs"]:
        res.append(operand(w, ng))
    return np.stack(res, axis=1)
