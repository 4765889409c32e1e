"""High-precision restatement of the pdf *definitions* in mpmath, used only to
pin the oracle.  Nothing here reuses the oracle's closed forms: every
normalisation is a numerical integral of the shape, and the Gauss (x) exp
decay shape is the convolution integral itself (paper Fig. 1: the signal is a
convolution of PDFs), not its erfc form.
"""
import mpmath as mp

mp.mp.dps = 30


def _params(nodes, node, theta):
    out = []
    for i in nodes[node].inputs[1:]:
        p = nodes[i]
        out.append(mp.mpf(theta[_free_index(nodes, i)]) if p.free else mp.mpf(p.value))
    return out


def _free_index(nodes, i):
    k = 0
    for j, n in enumerate(nodes):
        if j == i:
            return k
        if n.kind == "param" and n.free:
            k += 1
    raise IndexError


def _obs_column(nodes, i):
    return sum(1 for n in nodes[:i] if n.kind == "obs")


def shape(kind, x, q, a, b):
    x = mp.mpf(x)
    if kind == "gauss":
        mu, sg = q
        return mp.exp(-((x - mu) / sg) ** 2 / 2)
    if kind == "exp":
        return mp.exp(q[0] * x)
    if kind == "gaussexp":
        tau, mu, sg = q
        # f(t) = int_0^inf exp(-t'/tau) N(t - t'; mu, sg) dt'
        c = x - mu
        # Breakpoints where the integrand changes: around the Gaussian's centre
        # and, when the centre lies left of 0, geometrically from 0 on the
        # integrand's decay length sg^2/|c|.
        w = min(sg, sg * sg / abs(c)) if c != 0 else sg
        pts = {mp.mpf(0), max(mp.mpf(0), c - 12 * sg), max(mp.mpf(0), c), max(mp.mpf(0), c + 12 * sg)}
        pts |= {w * k / 4 for k in range(1, 40)}
        pts |= {w * 2 ** k for k in range(4, 14)}
        pts = sorted(pts) + [mp.inf]
        return mp.quad(lambda tp: mp.exp(-tp / tau) * mp.npdf(x - tp, mu, sg), pts)
    if kind == "cheb":
        xp = (2 * x - a - b) / (b - a)
        return 1 + sum(q[k] * mp.chebyt(k + 1, xp) for k in range(len(q)))
    if kind == "poly":
        return 1 + sum(q[k] * x ** (k + 1) for k in range(len(q)))
    raise ValueError(kind)


def expr_value(prog, consts, x, q):
    """The postfix program of an expr node at x, in mpmath (its own
    interpreter: code | arg << 8; x, parameter, constant pushes; + - * /
    pow pop two; neg exp log pop one)."""
    st = []
    for op in prog:
        code, arg = op & 0xFF, op >> 8
        if code == 0:
            st.append(mp.mpf(x))
        elif code == 1:
            st.append(q[arg])
        elif code == 2:
            st.append(mp.mpf(consts[arg]))
        elif code == 7:
            st.append(-st.pop())
        elif code == 8:
            st.append(mp.exp(st.pop()))
        elif code == 9:
            st.append(mp.log(st.pop()))
        else:
            bv, av = st.pop(), st.pop()
            st.append({3: av + bv, 4: av - bv, 5: av * bv, 6: av / bv, 10: av ** bv}[code])
    assert len(st) == 1
    return st[0]


def norm(kind, q, a, b):
    a, b = mp.mpf(a), mp.mpf(b)
    if kind == "gaussexp":
        tau, mu, sg = q
        # Fubini: int_a^b f = int_0^inf exp(-t'/tau) [Phi((b-t'-mu)/sg) - Phi((a-t'-mu)/sg)] dt'
        g = lambda tp: mp.exp(-tp / tau) * (mp.ncdf((b - tp - mu) / sg) - mp.ncdf((a - tp - mu) / sg))
        pts = sorted({mp.mpf(0), max(mp.mpf(0), a - mu), max(mp.mpf(0), b - mu)}) + [mp.inf]
        return mp.quad(g, pts)
    pts = [a, b]
    if kind == "gauss":
        mu = q[0]
        if a < mu < b:
            pts = [a, mu, b]
    return mp.quad(lambda t: shape(kind, t, q, a, b), pts)


def pdf(nodes, node, theta, x, _cache=None):
    """Normalised probability of `node` at event x (tuple over columns)."""
    n = nodes[node]
    if n.kind == "expr":
        ob = nodes[n.inputs[0]]
        q = _params(nodes, node, theta)
        key = (node, tuple(q))
        if _cache is not None and key in _cache:
            I = _cache[key]
        else:
            f = lambda t: expr_value(n.prog, n.consts, t, q)
            # split the range at 32 points so a narrow peak is resolved
            pts = [mp.mpf(ob.lo) + (mp.mpf(ob.hi) - mp.mpf(ob.lo)) * k / 32 for k in range(33)]
            I = mp.quad(f, pts)
            if _cache is not None:
                _cache[key] = I
        return expr_value(n.prog, n.consts, x[_obs_column(nodes, n.inputs[0])], q) / I
    if n.kind in ("gauss", "exp", "gaussexp", "cheb", "poly"):
        ob = nodes[n.inputs[0]]
        q = _params(nodes, node, theta)
        key = (node, tuple(q))
        if _cache is not None and key in _cache:
            I = _cache[key]
        else:
            I = norm(n.kind, q, ob.lo, ob.hi)
            if _cache is not None:
                _cache[key] = I
        return shape(n.kind, x[_obs_column(nodes, n.inputs[0])], q, ob.lo, ob.hi) / I
    if n.kind == "sum":
        nc = (len(n.inputs) + 1) // 2
        fr = []
        for i in n.inputs[nc:]:
            p = nodes[i]
            fr.append(mp.mpf(theta[_free_index(nodes, i)]) if p.free else mp.mpf(p.value))
        v = sum(fr[j] * pdf(nodes, n.inputs[j], theta, x, _cache) for j in range(nc - 1))
        return v + (1 - sum(fr)) * pdf(nodes, n.inputs[nc - 1], theta, x, _cache)
    if n.kind == "prod":
        v = mp.mpf(1)
        for c in n.inputs:
            v *= pdf(nodes, c, theta, x, _cache)
        return v
    raise ValueError(n.kind)


def nll(nodes, root, theta, events):
    """-sum log p over a few events, by the definitions, in 30-digit arithmetic."""
    cache = {}
    return -mp.fsum(mp.log(pdf(nodes, root, theta, ev, cache)) for ev in events)
