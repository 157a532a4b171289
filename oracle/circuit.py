"""Canonical gate netlist of the paper's encrypted FFT (oracle side).

The paper builds the FFT bottom-up from NAND-universal gates (Sec. 4,
Lemma 4), half and full adders (Lemmas 5-6, Fig. 3), ripple-carry addition
and subtraction by inverting the second operand with carry-in 1 (Sec. 4,
Lemma 7), Wallace-tree multiplication with sign extension and dropped high
bits (Lemma 8), the fixed-point "middle bits" of the product (Lemma 9), and
radix-2 butterflies after a plaintext bit reversal (Sec. 4, Lemma 3).

Each 2-input gate is one arithmetised GSW gate (codes in ``gsw.GATE_CODES``):
AND, XOR, OR each cost one ciphertext product, NOT is linear. The canonical
choices the paper leaves open (each a reading of the paper):

* Operand order. The product BitDecomp(A') B' is not symmetric in its
  ciphertext bits. A is the operand of strictly larger multiplicative depth,
  ties go to the gate's first argument. Depth: inputs and constants 0, a
  product gate 1 + max of its inputs, NOT the depth of its input.
* Constant folding. Gates with a trivial-constant input are replaced by their
  value (AND(x,1)=x, XOR(x,1)=NOT x, OR(x,1)=1, ...). In the compressed
  scheme these replacements are bit-exact (BitDecomp(P) = I, BitDecomp(A')P =
  A'), so folding never changes a ciphertext.
* HA(x,y) = (XOR(x,y), AND(x,y)); FA(x,y,z) = HA(x,y) -> (s1,c1),
  HA(s1,z) -> (s,c2), carry OR(c1,c2) (Lemma 6). Variant (``xcarry``): the
  two carries are never both 1 (c1 = 1 forces s1 = 0, hence c2 = 0), so the
  carry is their sum XADD(c1,c2), a linear gate with no product whose noise
  adds instead of growing by Ng; XADD folds like OR (x + 0 = x, and a
  constant 1 forces the other carry to 0, giving 1).
* ADD_F(x,y,cin): bit 0 is HA when cin is the constant 0, else FA; bits
  1..F-1 FA; carry out of the top bit dropped. SUB_F(x,y) = ADD_F(x, NOT y, 1).
* MUL(x, w) for a plaintext constant w, T = f + F: sign-extend x and w to T
  bits; each set bit i of w adds row i (column c >= i receives x_ext[c-i]),
  column lists in row order; Wallace stages until every column holds <= 2
  wires (per column: FAs on consecutive triples from the front, an HA on a
  remaining pair, a single wire passes; the new column is sums, then the
  passed wire, then carries from the column below; carries out of column
  T-1 dropped); then ADD_T of the two rows (missing wires = constant 0);
  result = bits [f, f+F). Closed form: floor(x w / 2^f) mod 2^F.
* Butterfly (Sec. 4; Sec. 5 eq. X_i = x_i + W x_j): t_r = SUB(MUL(x_r,Wr),
  MUL(x_i,Wi)); t_i = ADD(MUL(x_i,Wr), MUL(x_r,Wi)); top = u + t; bottom = u - t.
* FFT: iterative radix-2 decimation in time on the bit-reversed input, stage
  s = 1..log2 N with span m = 2^s and twiddle W_N^(j N/m); no 1/N scaling.
  2-D: every row, then every column.

Depth (for the operand rule): XADD, like NOT, is linear: the max of its inputs.

NAND-only variant (``nand``, the paper's literal construction, Lemma 4 and
Sec. 7's counts): constants fold first exactly as above; every remaining gate
is made of GSW NAND gates (one product each, code (1, 0, 0, -1)): NOT a =
NAND(a, a), AND = NOT(NAND(a, b)), OR = NAND(NOT a, NOT b), XOR =
NAND(NAND(a, t), NAND(b, t)) with t = NAND(a, b); a half adder shares t
between its XOR and its AND = NAND(t, t).

Encrypted-operand multiplier (``MULE``, a variant; the paper multiplies by
plaintext constants and notes in Sec. 4 that the constant's bits show through
the Wallace tree): both words are sign-extended to T = f + F bits and every
row i < T is present, column c >= i receiving AND(x_ext[c-i], y_ext[i]); the
same Wallace stages and final ADD_T as MUL; result bits [f, f+F). Closed form:
floor(x y / 2^f) mod 2^F. With ``enc_twiddle`` the FFT takes its twiddles as
encrypted words (inputs after the signal): one table W_M^k, k < M/2, M the
largest transform length, and a length-n transform uses entry t M/n for its
W_n^t (the same floor of the same real number).

Wires are non-negative ints; the trivial constants are ZERO = -1, ONE = -2.
Input wire number (k * 2 + part) * F + bit holds bit ``bit`` of the real
(part 0) or imaginary (part 1) word of sample k; with ``enc_twiddle`` sample
N1 N2 + k holds the twiddle W_M^k (real part Wr, imaginary part Wi).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import math

ZERO, ONE = -1, -2


class Circuit:
    def __init__(self, xcarry=False, nand=False):
        if xcarry and nand:
            raise ValueError("the NAND-only circuit has no linear carry")
        self.xcarry = xcarry   # full-adder carry as XADD instead of OR
        self.nand = nand       # every gate made of NAND gates
        self.gates = []      # (op, a, b, out); b is None for NOT
        self.depth = []      # per wire
        self.inputs = []
        self.outputs = []

    # -- wires -------------------------------------------------------------
    def new_input(self):
        w = len(self.depth)
        self.depth.append(0)
        self.inputs.append(w)
        return w

    def d(self, w):
        return 0 if w < 0 else self.depth[w]

    def _emit(self, op, a, b, depth):
        w = len(self.depth)
        self.depth.append(depth)
        self.gates.append((op, a, b, w))
        return w

    # -- gates with constant folding (Lemma 4) -----------------------------
    def _nand(self, a, b):
        """A GSW NAND gate on two non-constant wires (NAND-only variant; the
        scheme's own gate, Sec. 3, from which Lemma 4 builds the others)."""
        return self._emit("NAND", a, b, 1 + max(self.d(a), self.d(b)))

    def NOT(self, a):
        if a == ZERO:
            return ONE
        if a == ONE:
            return ZERO
        if self.nand:
            return self._nand(a, a)
        return self._emit("NOT", a, None, self.d(a))

    def AND(self, a, b):
        if a == ZERO or b == ZERO:
            return ZERO
        if a == ONE:
            return b
        if b == ONE:
            return a
        if self.nand:
            return self.NOT(self._nand(a, b))
        return self._emit("AND", a, b, 1 + max(self.d(a), self.d(b)))

    def XOR(self, a, b):
        if a == ZERO:
            return b
        if b == ZERO:
            return a
        if a == ONE:
            return self.NOT(b)
        if b == ONE:
            return self.NOT(a)
        if self.nand:
            t = self._nand(a, b)
            return self._nand(self._nand(a, t), self._nand(b, t))
        return self._emit("XOR", a, b, 1 + max(self.d(a), self.d(b)))

    def OR(self, a, b):
        if a == ONE or b == ONE:
            return ONE
        if a == ZERO:
            return b
        if b == ZERO:
            return a
        if self.nand:
            return self._nand(self.NOT(a), self.NOT(b))
        return self._emit("OR", a, b, 1 + max(self.d(a), self.d(b)))

    def XADD(self, a, b):
        """Sum of two bits that are never both 1 (linear)."""
        if a == ONE or b == ONE:
            return ONE
        if a == ZERO:
            return b
        if b == ZERO:
            return a
        return self._emit("XADD", a, b, max(self.d(a), self.d(b)))

    def SEL(self, a, beta):
        """beta * a for a public bit beta: a linear gate that is never folded
        (its structure must not depend on beta; refresh circuits, the
        refreshing Sec. 5 points at)."""
        return self._emit("SEL1" if beta else "SEL0", a, None, self.d(a))

    # -- adders (Lemmas 5-7) ---------------------------------------------
    def HA(self, a, b):
        if self.nand and a not in (ZERO, ONE) and b not in (ZERO, ONE):
            t = self._nand(a, b)
            return self._nand(self._nand(a, t), self._nand(b, t)), self._nand(t, t)
        return self.XOR(a, b), self.AND(a, b)

    def FA(self, a, b, c):
        s1, c1 = self.HA(a, b)
        s, c2 = self.HA(s1, c)
        return s, (self.XADD(c1, c2) if self.xcarry else self.OR(c1, c2))

    def ADD(self, x, y, cin=ZERO):
        F = len(x)
        out = []
        if cin == ZERO:
            s, c = self.HA(x[0], y[0])
        else:
            s, c = self.FA(x[0], y[0], cin)
        out.append(s)
        for i in range(1, F):
            s, c = self.FA(x[i], y[i], c)
            out.append(s)
        return out   # final carry dropped (wraps mod 2^F)

    def SUB(self, x, y):
        return self.ADD(x, [self.NOT(b) for b in y], ONE)

    # -- Wallace constant multiplier (Lemmas 8-9) --------------------------
    def MUL(self, x, w, f):
        F = len(x)
        T = f + F
        x_ext = [x[min(j, F - 1)] for j in range(T)]
        w_bits = w % (1 << T)
        cols = [[] for _ in range(T)]
        for i in range(T):
            if (w_bits >> i) & 1:
                for c in range(i, T):
                    cols[c].append(x_ext[c - i])
        return self._wallace(cols)[f:f + F]

    def MULE(self, x, y, f):
        """Fixed-point product of two encrypted words (AND partial products):
        Lemma 8's sign-extended Wallace product with every row present,
        Lemma 9's middle bits (the encrypted-operand case Sec. 4 mentions
        beside constant multiplication)."""
        F = len(x)
        T = f + F
        x_ext = [x[min(j, F - 1)] for j in range(T)]
        y_ext = [y[min(i, F - 1)] for i in range(T)]
        cols = [[] for _ in range(T)]
        for i in range(T):
            for c in range(i, T):
                cols[c].append(self.AND(x_ext[c - i], y_ext[i]))
        return self._wallace(cols)[f:f + F]

    def _wallace(self, cols):
        """Wallace stages on column lists, then ADD_T of the two rows (T bits);
        Lemma 8 with the stage rule stated in this module's docstring."""
        T = len(cols)
        while max(len(col) for col in cols) > 2:
            sums = [[] for _ in range(T)]
            passed = [[] for _ in range(T)]
            carries = [[] for _ in range(T + 1)]
            for c in range(T):
                col = cols[c]
                g = 0
                while len(col) - g >= 3:
                    s, cy = self.FA(col[g], col[g + 1], col[g + 2])
                    sums[c].append(s)
                    carries[c + 1].append(cy)
                    g += 3
                if len(col) - g == 2:
                    s, cy = self.HA(col[g], col[g + 1])
                    sums[c].append(s)
                    carries[c + 1].append(cy)
                elif len(col) - g == 1:
                    passed[c].append(col[g])
            cols = [sums[c] + passed[c] + carries[c] for c in range(T)]
        row0 = [col[0] if len(col) >= 1 else ZERO for col in cols]
        row1 = [col[1] if len(col) >= 2 else ZERO for col in cols]
        return self.ADD(row0, row1, ZERO)

    # -- butterfly and FFT (Sec. 4, Lemma 3) -------------------------------
    def BUTTERFLY(self, u, x, W, f):
        """W = (Wr, Wi): plaintext ints (MUL) or encrypted words (MULE)."""
        (ur, ui), (xr, xi), (Wr, Wi) = u, x, W
        mul = self.MULE if isinstance(Wr, list) else self.MUL
        tr = self.SUB(mul(xr, Wr, f), mul(xi, Wi, f))
        ti = self.ADD(mul(xi, Wr, f), mul(xr, Wi, f))
        top = (self.ADD(ur, tr), self.ADD(ui, ti))
        bot = (self.SUB(ur, tr), self.SUB(ui, ti))
        return top, bot

    def FFT(self, samples, tw, f):
        """Radix-2 DIT over a list of complex words; tw[k] = (Wr, Wi), k < N/2."""
        N = len(samples)
        logN = N.bit_length() - 1
        a = [samples[bitrev(i, logN)] for i in range(N)]
        m = 2
        while m <= N:
            h = m // 2
            for k in range(0, N, m):
                for j in range(h):
                    top, bot = self.BUTTERFLY(a[k + j], a[k + j + h], tw[j * (N // m)], f)
                    a[k + j], a[k + j + h] = top, bot
            m *= 2
        return a

    # -- dead code ------------------------------------------------------------
    def prune(self):
        """Drop gates whose outputs reach no circuit output (bit-neutral)."""
        live = set(w for w in self.outputs if w >= 0)
        kept = []
        for g in reversed(self.gates):
            op, a, b, o = g
            if o in live:
                kept.append(g)
                live.add(a)
                if b is not None:
                    live.add(b)
        kept.reverse()
        self.gates = kept


def bitrev(i, bits):
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


def twiddles(N, f):
    """W_N^k = exp(-2 pi i k / N) quantised by floor to 2^-f, k < N/2."""
    tw = []
    for k in range(N // 2):
        ang = 2.0 * math.pi * k / N
        tw.append((math.floor(math.cos(ang) * (1 << f)), math.floor(-math.sin(ang) * (1 << f))))
    return tw


def fft_circuit(N1, N2, F, f, xcarry=False, nand=False, enc_twiddle=False):
    """Circuit of a 1-D (N2 == 1) or row-column 2-D encrypted FFT.

    1-D: N1 samples. 2-D: an N1 x N2 image, sample k = r * N2 + c; all row
    FFTs (length N2) first, then all column FFTs (length N1). ``xcarry``
    selects the exclusive-carry full adder, ``nand`` the NAND-only gates,
    ``enc_twiddle`` encrypted twiddle inputs (needs f <= F - 2 so that
    W_M^0 = 2^f fits a signed F-bit word).
    """
    for n in (N1, N2):
        if n < 1 or n & (n - 1):
            raise ValueError("FFT sizes must be powers of two")
    if enc_twiddle and f > F - 2:
        raise ValueError("encrypted twiddles need f <= F - 2")
    c = Circuit(xcarry, nand)
    count = N1 * N2
    samples = []
    for k in range(count):
        re = [c.new_input() for _ in range(F)]
        im = [c.new_input() for _ in range(F)]
        samples.append((re, im))
    M = max(N1, N2)
    if enc_twiddle:
        table = []
        for k in range(M // 2):
            wr = [c.new_input() for _ in range(F)]
            wi = [c.new_input() for _ in range(F)]
            table.append((wr, wi))

        def tw_of(n):
            return [table[t * (M // n)] for t in range(n // 2)]
    else:
        def tw_of(n):
            return twiddles(n, f)
    if N2 == 1:
        out = c.FFT(samples, tw_of(N1), f) if N1 > 1 else samples
    else:
        rows = [c.FFT(samples[r * N2:(r + 1) * N2], tw_of(N2), f) if N2 > 1
                else samples[r * N2:(r + 1) * N2] for r in range(N1)]
        grid = [x for row in rows for x in row]
        out = list(grid)
        if N1 > 1:
            tw = tw_of(N1)
            for col in range(N2):
                res = c.FFT([grid[r * N2 + col] for r in range(N1)], tw, f)
                for r in range(N1):
                    out[r * N2 + col] = res[r]
    for re, im in out:
        c.outputs.extend(re)
        c.outputs.extend(im)
    c.prune()
    return c


def word_circuit(kind, F, f=0, w=None, xcarry=False, nand=False):
    """Small circuits over two input words (x, y) for the arithmetic pins.

    kind: 'add', 'sub' (x op y), 'mul' (x times plaintext w, fixed point f),
    'mule' (x times the encrypted y, fixed point f).
    """
    c = Circuit(xcarry, nand)
    x = [c.new_input() for _ in range(F)]
    y = [c.new_input() for _ in range(F)]
    if kind == "add":
        out = c.ADD(x, y)
    elif kind == "sub":
        out = c.SUB(x, y)
    elif kind == "mul":
        out = c.MUL(x, w, f)
    elif kind == "mule":
        out = c.MULE(x, y, f)
    else:
        raise ValueError(kind)
    c.outputs = list(out)
    c.prune()
    return c


def stats(c):
    """Counts of each gate kind and of ciphertext products (AND/XOR/OR;
    XADD, NOT and SEL are linear)."""
    s = {"NOT": 0, "AND": 0, "XOR": 0, "OR": 0, "XADD": 0, "NAND": 0, "SEL0": 0, "SEL1": 0}
    for op, *_ in c.gates:
        s[op] += 1
    # One product per distinct (kind, A, B) after value numbering: an HA's XOR
    # and AND share it, and identical gates (e.g. the repeated sign-extension
    # columns of a Wallace tree) compute identical ciphertexts. A wire's value
    # number is (base wire, complemented?) so that NOT(NOT x) is x.
    canon = {ZERO: (ZERO, 0), ONE: (ZERO, 1)}
    for w in c.inputs:
        canon[w] = (w, 0)
    seen = {}
    pairs = set()
    for op, a, b, o in c.gates:
        if op == "NOT":
            base, neg = canon[a]
            canon[o] = (base, 1 - neg)
            continue
        if op in ("SEL0", "SEL1"):    # distinct wires whatever their source
            canon[o] = (o, 0)
            continue
        A, B = (b, a) if c.d(b) > c.d(a) else (a, b)
        key = (op, canon[A], canon[B])
        if key not in seen:
            seen[key] = (o, 0)
        canon[o] = seen[key]
        if op != "XADD":
            pairs.add((op if op in ("OR", "NAND") else "HA", canon[A], canon[B]))
    s["products"] = len(pairs)
    s["depth"] = max((c.depth[o] for _, _, _, o in c.gates), default=0)
    return s
