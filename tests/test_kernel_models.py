"""CPU models of the index and bit-level logic of five CUDA kernels (no GPU).

Each model repeats in Python, step by step, what one kernel does with its
data -- which boxes it stages into which ring slot, which lane or row hands a
value to which, which integer operations it applies to IEEE bit patterns --
and is compared with the plain definition of the same result:

* k_cc_rb_sweep (solvers.cu), one red-black Gauss-Seidel sweep in one pass
  (paper Sec. "Numerical algorithm": red-black Gauss-Seidel smoothing of the
  multigrid solves): the TMA boxes with zero fill, the plane rings, the first
  colour on the tile and its one-cell ring, the second colour one plane
  behind, the staged coarse correction of the sweep after the coarse-grid
  correction and the r.z partials, against two colour passes; every staged
  read must come from the slot that holds the plane it wants, every index
  must lie inside its box (the first colour is modelled cell by cell, where
  the kernel pairs its shared-memory loads; the second colour in pairs);
* k_slopes_march (fields.cu): the face differences handed on by lane shuffle,
  shared row and register, against the direct differences, bit for bit;
* mc_limit (fields.cu): the monotonised-central limiter on the 32-bit words of
  the IEEE patterns, against the same limiter on 64-bit patterns;
* k_cc_rr4 (solvers.cu): residual and restriction with 4-wide vectors,
  against the residuals of the first-colour children averaged one by one;
* k_cc_gs2_dot (solvers.cu): the last colour pass forming the fused sweep's
  (plane, tile) partials of b.x, against the fused sweep's own.

These are models of the kernels' logic, not the kernels; the GPU tests
compare the kernels with the oracle.
"""
import itertools
import math
import random
import struct

import numpy as np
import pytest

# ---- k_cc_rb_sweep --------------------------------------------------------
HW, TY = 32, 16                    # tile: half-row positions, rows
XW, FW = HW + 8, HW + 16           # box widths: cells (4 each side), faces (8 each side)
XR, CR, YR = TY + 4, TY + 2, TY + 3
KW, KR = 24, TY // 2 + 2           # coarse box
THREADS = 256


class Grid:
    def __init__(self, nx, ny, nz):
        self.nx, self.ny, self.nz = nx, ny, nz


def cix(g, i, j, k):
    """Row-split index: even cells of a row, then odd ones (nx even)."""
    return (k * g.ny + j) * g.nx + ((g.nx >> 1) + (i >> 1) if i & 1 else i >> 1)


def colour_passes(g, b, dinv, x, bx, by, bz, c0, zero, xc=None, gc=None):
    """Two colour passes: colour c0 (neighbours plus the parents' coarse
    correction when xc is given), then colour 1 - c0."""
    x = np.zeros_like(x) if zero else x.copy()
    hf = (g.nx + 2) >> 1

    def cell(i, j, k, corr):
        c = cix(g, i, j, k)
        t, odd = i >> 1, i & 1
        rf = (k * g.ny + j) * (g.nx + 1)
        bxl = bx[rf + (hf + t if odd else t)]
        bxh = bx[rf + (t + 1 if odd else hf + t)]
        fy0, fy1 = by[c + k * g.nx], by[c + k * g.nx + g.nx]
        fz0, fz1 = bz[c], bz[c + g.nx * g.ny]

        def X(ii, jj, kk):
            v = x[cix(g, ii, jj, kk)]
            return v + xc[cix(gc, ii >> 1, jj >> 1, kk >> 1)] if corr else v
        s = 0.0
        if i > 0: s += bxl * X(i - 1, j, k)
        if i < g.nx - 1: s += bxh * X(i + 1, j, k)
        if j > 0: s += fy0 * X(i, j - 1, k)
        if j < g.ny - 1: s += fy1 * X(i, j + 1, k)
        if k > 0: s += fz0 * X(i, j, k - 1)
        if k < g.nz - 1: s += fz1 * X(i, j, k + 1)
        return (b[c] + s) * dinv[c]

    for col, corr in ((c0, xc is not None), (1 - c0, False)):
        new = {cix(g, i, j, k): cell(i, j, k, corr)
               for k in range(g.nz) for j in range(g.ny) for i in range(g.nx) if (i + j + k) & 1 == col}
        for c, v in new.items():
            x[c] = v
    return x


class Box:
    """A 4-D TMA box (half-row position, half, row, plane) with zero fill."""

    def __init__(self, arr, hx, rows_total, planes_total, width, rows):
        self.arr, self.hx, self.R, self.P, self.w, self.rows = arr, hx, rows_total, planes_total, width, rows

    def load(self, p0, r0, plane):
        out = np.zeros(self.rows * 2 * self.w)
        for r in range(self.rows):
            for h in range(2):
                for q in range(self.w):
                    p, row = p0 + q, r0 + r
                    if 0 <= p < self.hx and 0 <= row < self.R and 0 <= plane < self.P:
                        out[(r * 2 + h) * self.w + q] = self.arr[(plane * self.R + row) * 2 * self.hx + h * self.hx + p]
        return out


def fused_sweep(g, b, dinv, xin, bx, by, bz, c0, mode, xc=None, gc=None, kz=None):
    """The fused sweep (mode 0 from zero, 1 plain, 2 after the coarse
    correction, 3 with r.z partials), block by block and step by step."""
    hx, hf = g.nx >> 1, (g.nx + 2) >> 1
    zero, corr, dot = mode == 0, mode == 2, mode == 3
    xout = np.full(g.nx * g.ny * g.nz, np.nan)
    kz = kz or g.nz
    part = {}
    BX = Box(xin, hx, g.ny, g.nz, XW, XR)
    BB = Box(b, hx, g.ny, g.nz, XW, CR)
    BD = Box(dinv, hx, g.ny, g.nz, XW, CR)
    BY = Box(by, hx, g.ny + 1, g.nz, FW, YR)
    BZ = Box(bz, hx, g.ny, g.nz + 1, FW, CR)
    hxp = ((g.nx // 2 + 1) + 7) // 8 * 8          # the padded x-face copy
    bxp = np.zeros(2 * hxp * g.ny * g.nz)
    for row in range(g.ny * g.nz):
        rf = row * (g.nx + 1)
        for pos in range(hxp):
            if pos < hf: bxp[row * 2 * hxp + pos] = bx[rf + pos]
            if pos < hx: bxp[(row * 2 + 1) * hxp + pos] = bx[rf + hf + pos]
    BXF = Box(bxp, hxp, g.ny, g.nz, FW, CR)
    if corr:
        BK = Box(xc, gc.nx >> 1, gc.ny, gc.nz, KW, KR)
    c1 = 1 - c0
    for bxi, byi, bzi in itertools.product(range((hx + HW - 1) // HW), range((g.ny + TY - 1) // TY),
                                          range((g.nz + kz - 1) // kz)):
        p0, y0, z0 = bxi * HW, byi * TY, bzi * kz
        z1 = min(g.nz, z0 + kz)
        if z0 >= z1:
            continue
        assert (p0 - 4) * 4 % 16 == 0 and (p0 - 8) * 2 % 16 == 0 and (p0 // 2 - 4) * 4 % 16 == 0
        ring = {n: {} for n in ("X", "B", "D", "Y", "Z", "XF", "R", "K")}
        m0, nstep = z0 - 1, z1 - z0 + 2

        def put(name, slot, plane, data):
            ring[name][slot] = (plane, data)

        def get(name, slot, plane):
            held, data = ring[name][slot]
            assert held == plane, (name, held, plane)   # no slot overwritten before its last read
            return data

        def issue(q):
            m = m0 + q
            if corr:
                nk = 2 if q == 0 else (1 if (m + 1) % 2 == 0 else 0)
                first = (m - 1) >> 1 if q == 0 else (m + 1) >> 1
                for t in range(nk):
                    C = first + t
                    put("K", (C + 3) % 3, C, BK.load(p0 // 2 - 4, y0 // 2 - 1, C))
            if not zero:
                for pl in ((m - 1, m, m + 1) if q == 0 else (m + 1,)):
                    put("X", (pl + 8) & 3, pl, BX.load(p0 - 4, y0 - 2, pl))
            s = (m + 3) % 3
            put("B", s, m, BB.load(p0 - 4, y0 - 1, m))
            put("D", s, m, BD.load(p0 - 4, y0 - 1, m))
            put("Y", s, m, BY.load(p0 - 8, y0 - 1, m))
            put("XF", s, m, BXF.load(p0 - 8, y0 - 1, m))
            for pl in ((m, m + 1) if q == 0 else (m + 1,)):
                put("Z", (pl + 8) & 3, pl, BZ.load(p0 - 8, y0 - 1, pl))

        X = lambda pl: get("X", (pl + 8) & 3, pl)
        B = lambda pl: get("B", (pl + 3) % 3, pl)
        D = lambda pl: get("D", (pl + 3) % 3, pl)
        FY = lambda pl: get("Y", (pl + 3) % 3, pl)
        FXF = lambda pl: get("XF", (pl + 3) % 3, pl)
        FZ = lambda pl: get("Z", (pl + 8) & 3, pl)
        R = lambda pl: get("R", (pl + 3) % 3, pl)

        def parents(k, j, p, h):
            """The four distinct coarse values around cell (2p + h, j, k): its
            parent, and per axis the next coarse cell on the neighbour's side."""
            Kk, Ko = get("K", ((k >> 1) + 3) % 3, k >> 1), (k >> 1) - 1 + 2 * (k & 1)
            Kop = get("K", (Ko + 3) % 3, Ko)
            J, Jo = j >> 1, (j >> 1) - 1 + 2 * (j & 1)
            row = lambda jj: (jj - (y0 // 2 - 1)) * 2 * KW
            col = lambda I: (I & 1) * KW + (I >> 1) - (p0 // 2 - 4)
            for jj, I in ((J, p), (Jo, p), (J, p + 1 if h else p - 1)):
                assert 0 <= row(jj) // (2 * KW) < KR and 0 <= col(I) - (I & 1) * KW < KW
            co, cx = Kk[row(J) + col(p)], Kk[row(J) + col(p + 1 if h else p - 1)]
            cy, cz = Kk[row(Jo) + col(p)], Kop[row(J) + col(p)]
            return co, cx, cy, cz

        issue(0)
        issue(1)
        for q in range(nstep):
            m = m0 + q
            if 0 <= m < g.nz:
                # first colour on plane m: tile and one-cell ring, into R(m)
                Rm = np.full(CR * XW, np.nan)
                Bm, Dm, Fy, Fz0, Fz1, Fx = B(m), D(m), FY(m), FZ(m), FZ(m + 1), FXF(m)
                X0, X1, X2 = (X(m - 1), X(m), X(m + 1)) if not zero else (None, None, None)

                def first(r1, j, h, p):
                    i, k, qx, qf = 2 * p + h, m, p - p0 + 4, p - p0 + 8
                    assert 0 <= qx - 1 and qx + 1 < XW and 0 <= qf and qf + 1 < FW and 0 <= r1 < CR
                    cc = (r1 * 2 + h) * XW + qx
                    off = 0.0
                    if not zero:
                        rx = r1 + 1
                        xi = lambda Xp, rr, hh, qq: Xp[(rr * 2 + hh) * XW + qq]
                        xw = xi(X1, rx, 0, qx) if h else xi(X1, rx, 1, qx - 1)
                        xe = xi(X1, rx, 0, qx + 1) if h else xi(X1, rx, 1, qx)
                        xs, xn = xi(X1, rx - 1, h, qx), xi(X1, rx + 1, h, qx)
                        xd, xu = xi(X0, rx, h, qx), xi(X2, rx, h, qx)
                        if corr:
                            co, cx, cy, cz = parents(k, j, p, h)
                            if i > 0: xw += co if h else cx
                            if i < g.nx - 1: xe += cx if h else co
                            if j > 0: xs += co if j & 1 else cy
                            if j < g.ny - 1: xn += cy if j & 1 else co
                            if k > 0: xd += co if k & 1 else cz
                            if k < g.nz - 1: xu += cz if k & 1 else co
                        if i > 0: off += Fx[(r1 * 2 + h) * FW + qf] * xw
                        if i < g.nx - 1: off += Fx[(r1 * 2 + 1 - h) * FW + qf + h] * xe
                        if j > 0: off += Fy[(r1 * 2 + h) * FW + qf] * xs
                        if j < g.ny - 1: off += Fy[((r1 + 1) * 2 + h) * FW + qf] * xn
                        if k > 0: off += Fz0[(r1 * 2 + h) * FW + qf] * xd
                        if k < g.nz - 1: off += Fz1[(r1 * 2 + h) * FW + qf] * xu
                    Rm[r1 * XW + qx] = (Bm[cc] + off) * Dm[cc]    # only the first colour's half

                for tid in range(THREADS):
                    r, pq = tid >> 4, p0 + 2 * (tid & 15)
                    j = y0 + r
                    if j < g.ny and pq < hx:
                        for e in range(2):
                            first(r + 1, j, (c0 + j + m) & 1, pq + e)
                    t = tid // 3                                    # the ring on every third thread
                    if tid % 3 == 0 and t < 2 * (HW + 1) + TY:
                        w = t if t < HW + 1 else t - (HW + 1)
                        if t < 2 * (HW + 1):
                            r1 = 0 if t < HW + 1 else CR - 1
                            jj = y0 - 1 + r1
                            pp = (p0 - 1 if (c0 + jj + m) & 1 else p0) + w
                        else:
                            r1 = t - 2 * (HW + 1) + 1
                            jj = y0 - 1 + r1
                            pp = p0 - 1 if (c0 + jj + m) & 1 else p0 + HW
                        if 0 <= jj < g.ny and 0 <= pp < hx:
                            first(r1, jj, (c0 + jj + m) & 1, pp)
                put("R", (m + 3) % 3, m, Rm)
            mm = m - 1
            if q >= 2:
                # second colour on plane mm from the first colour's results, and the output
                Rc = R(mm)
                Rl = R(mm - 1) if mm > 0 else None
                Rh = R(mm + 1) if mm + 1 < g.nz else None
                Bm, Dm, Fy, Fz0, Fz1, Fx = B(mm), D(mm), FY(mm), FZ(mm), FZ(mm + 1), FXF(mm)
                for tid in range(THREADS):
                    r, pq = tid >> 4, p0 + 2 * (tid & 15)
                    j = y0 + r
                    if not (j < g.ny and pq < hx):
                        continue
                    rc, qx, hh, k = r + 1, pq - p0 + 4, (c1 + j + mm) & 1, mm
                    qf, ch, cr = qx + 4, (rc * 2 + hh) * XW + qx, rc * XW + qx
                    assert cr - XW >= 0 and cr + XW + 1 < CR * XW and cr - 1 >= 0 and cr + 2 < CR * XW
                    xo = Rc[cr:cr + 2]
                    xb = Rc[cr + 2] if hh else Rc[cr - 1]
                    xw2 = [xo[0] if hh else xb, xo[1] if hh else xo[0]]
                    xe2 = [xo[1] if hh else xo[0], xb if hh else xo[1]]
                    s2 = [0.0, 0.0]
                    for e in range(2):
                        i = 2 * (pq + e) + hh
                        off = 0.0
                        if i > 0: off += Fx[(rc * 2 + hh) * FW + qf + e] * xw2[e]
                        if i < g.nx - 1: off += Fx[(rc * 2 + 1 - hh) * FW + qf + hh + e] * xe2[e]
                        if j > 0: off += Fy[(rc * 2 + hh) * FW + qf + e] * Rc[cr - XW + e]
                        if j < g.ny - 1: off += Fy[((rc + 1) * 2 + hh) * FW + qf + e] * Rc[cr + XW + e]
                        if k > 0: off += Fz0[(rc * 2 + hh) * FW + qf + e] * Rl[cr + e]
                        if k < g.nz - 1: off += Fz1[(rc * 2 + hh) * FW + qf + e] * Rh[cr + e]
                        assert not np.isnan(off)
                        s2[e] = (Bm[ch + e] + off) * Dm[ch + e]
                    v = [[xo[e] if hh else s2[e] for e in range(2)], [s2[e] if hh else xo[e] for e in range(2)]]
                    o = (mm * g.ny + j) * g.nx + pq
                    xout[o:o + 2] = v[0]
                    xout[o + hx:o + hx + 2] = v[1]
                    if dot:
                        key = (mm, byi, bxi)
                        part[key] = part.get(key, 0.0) + sum(Bm[(rc * 2 + h) * XW + qx + e] * v[h][e]
                                                             for h in range(2) for e in range(2))
            if q + 2 < nstep:
                issue(q + 2)
    return xout, part


@pytest.mark.parametrize("shape,kz", [((16, 5, 3), 2), ((32, 17, 5), 2), ((80, 20, 4), 3), ((48, 18, 7), 7)])
def test_rb_sweep_model_matches_colour_passes(shape, kz):
    g = Grid(*shape)
    rng = np.random.default_rng(1)
    n = g.nx * g.ny * g.nz
    b, dinv, x = rng.standard_normal(n), rng.uniform(0.1, 0.3, n), rng.standard_normal(n)
    bx = rng.uniform(0, 1, (g.nx + 1) * g.ny * g.nz)
    by = rng.uniform(0, 1, g.nx * (g.ny + 1) * g.nz)
    bz = rng.uniform(0, 1, g.nx * g.ny * (g.nz + 1))
    gc = Grid((g.nx + 1) // 2, (g.ny + 1) // 2, (g.nz + 1) // 2)
    xc = rng.standard_normal(gc.nx * gc.ny * gc.nz)
    for c0 in (0, 1):
        for mode in range(4):
            cor = xc if mode == 2 else None
            ref = colour_passes(g, b, dinv, x, bx, by, bz, c0, mode == 0, cor, gc)
            out, part = fused_sweep(g, b, dinv, x, bx, by, bz, c0, mode, cor, gc, kz)
            assert not np.isnan(out).any(), "a cell was not written"
            assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max(), (c0, mode)
            if mode == 3:
                assert abs(sum(part.values()) - b @ ref) <= 1e-9 * abs(b @ ref)


# ---- k_slopes_march -------------------------------------------------------
SX, SY, SZ = 32, 8, 16


@pytest.mark.parametrize("shape", [(40, 11, 19), (32, 8, 16), (5, 3, 2), (70, 17, 33)])
def test_slope_march_hands_on_the_same_differences(shape):
    nx, ny, nz = shape
    rnd = random.Random(sum(shape))
    N3 = nx * ny * nz
    u = [rnd.uniform(-1, 1) for _ in range(3 * N3)]
    cidx = lambda i, j, k: (k * ny + j) * nx + i
    seen = set()
    for bx, by, bz in itertools.product(range((nx + SX - 1) // SX), range((ny + SY - 1) // SY),
                                        range((nz + SZ - 1) // SZ)):
        z0, z1 = bz * SZ, min(nz, bz * SZ + SZ)
        carry, shared = {}, {}
        for k in range(z0, z1):
            st = {}
            for ty, tx in itertools.product(range(SY), range(SX)):
                i, j = bx * SX + tx, by * SY + ty
                col = i < nx and j < ny
                c = cidx(i, j, k) if col else 0
                f0 = [u[q * N3 + c] if col else 0.0 for q in range(3)]
                drx = [u[q * N3 + c + 1] - f0[q] if col and i < nx - 1 else 0.0 for q in range(3)]
                dry = [u[q * N3 + c + nx] - f0[q] if col and j < ny - 1 else 0.0 for q in range(3)]
                drz = [u[q * N3 + c + nx * ny] - f0[q] if col and k < nz - 1 else 0.0 for q in range(3)]
                st[tx, ty] = (i, j, col, c, f0, drx, dry, drz)
                for q in range(3):
                    shared[k & 1, q, ty, tx] = dry[q]
            for ty, tx in itertools.product(range(SY), range(SX)):
                i, j, col, c, f0, drx, dry, drz = st[tx, ty]
                for q in range(3):
                    f = lambda idx: u[q * N3 + idx]
                    dlx = st[tx - 1, ty][5][q] if tx > 0 else drx[q]          # shuffle up (lane 0 keeps its own)
                    if tx == 0 and col and i > 0:
                        dlx = f0[q] - f(c - 1)
                    dly = shared[k & 1, q, ty - 1, tx] if ty > 0 else (f0[q] - f(c - nx) if col and j > 0 else 0.0)
                    dlz = carry[tx, ty, q] if k > z0 else (f0[q] - f(c - nx * ny) if col and k > 0 else 0.0)
                    carry[tx, ty, q] = drz[q]
                    if not col:
                        continue
                    if i > 0: assert dlx == f(c) - f(c - 1)
                    if i < nx - 1: assert drx[q] == f(c + 1) - f(c)
                    if j > 0: assert dly == f(c) - f(c - nx)
                    if k > 0: assert dlz == f(c) - f(c - nx * ny)
                    seen.add((q, c))
    assert len(seen) == 3 * N3


# ---- mc_limit on 32-bit words ---------------------------------------------
def _bits(x):
    return struct.unpack("<q", struct.pack("<d", x))[0]


def _limit64(dl, dr, dd):
    """The limiter on 64-bit patterns (the definition the 32-bit form keeps)."""
    kabs, ke = 0x7FFFFFFFFFFFFFFF, 1 << 52
    bl, br, bd = _bits(dl), _bits(dr), _bits(dd)
    al, ar, ad = bl & kabs, br & kabs, bd & kabs
    if al == 0 or ar == 0 or (bl ^ br) < 0:
        return ("zero",)
    lo, hi = 3 * ke, 2044 * ke
    if al < lo or ar < lo or (ad != 0 and ad < lo) or al >= hi or ar >= hi or ad >= hi:
        return ("fp64",)
    m4 = min(ad, al + 2 * ke, ar + 2 * ke)
    m = 0 if m4 == 0 else m4 - ke
    return ("bits", m if bd > 0 else m | (1 << 63))


def _limit32(dl, dr, dd):
    """The same on (high, low) 32-bit words, as mc_limit forms it."""
    def words(x):
        u = _bits(x) & 0xFFFFFFFFFFFFFFFF
        return u >> 32, u & 0xFFFFFFFF
    (lh, ll), (rh, rl), (dh, dlo) = words(dl), words(dr), words(dd)
    ks, ke1 = 0x80000000, 1 << 20
    alh, arh, adh = lh & ~ks, rh & ~ks, dh & ~ks
    if (alh | ll) == 0 or (arh | rl) == 0 or (lh ^ rh) & ks:
        return ("zero",)
    lo, hi = 3 * ke1, 2044 * ke1
    if alh < lo or arh < lo or ((adh | dlo) != 0 and adh < lo) or alh >= hi or arh >= hi or adh >= hi:
        return ("fp64",)
    mh, ml = alh + 2 * ke1, ll
    bh = arh + 2 * ke1
    if bh < mh or (bh == mh and rl < ml):
        mh, ml = bh, rl
    if adh < mh or (adh == mh and dlo < ml):
        mh, ml = adh, dlo
    if mh | ml:
        mh -= ke1
    pos = not (dh & ks) and (dh | dlo) != 0
    return ("bits", ((mh if pos else mh | ks) << 32) | ml)


def test_limiter_words_match_64bit_patterns():
    rnd = random.Random(5)
    special = [0.0, -0.0, 1.0, -1.0, 5e-324, -5e-324, 1e-310, 2.2250738585072014e-308, 1e308, -1e308,
               3.0, 3.0000000000000004, 0.75, 0.7500000000000001]

    def draw():
        c = rnd.random()
        if c < 0.15:
            return rnd.choice(special)
        if c < 0.3:
            return rnd.uniform(-2, 2)
        return rnd.choice([1, -1]) * math.ldexp(rnd.random() + 0.5, rnd.randint(-1070, 1023))

    for _ in range(40000):
        dl, dr = draw(), draw()
        c = rnd.random()
        dd = dl + dr if c < 0.3 else (0.0 if c < 0.4 else (-0.0 if c < 0.5 else draw()))
        if c > 0.9 and _bits(dl) >= 0:   # equal high words, different low words
            dr = struct.unpack("<d", struct.pack("<q", (_bits(dl) & ~0xFFFFFFFF) | rnd.getrandbits(32)))[0]
        if math.isinf(dd) or math.isnan(dd):
            continue
        a, b = _limit64(dl, dr, dd), _limit32(dl, dr, dd)
        if a[0] == "bits":
            a = ("bits", a[1] & 0xFFFFFFFFFFFFFFFF)
        assert a == b, (dl, dr, dd, a, b)


# ---- k_cc_rr4: residual and restriction, four coarse cells per thread -----
def _split_pos(m, i):
    return ((m + 1) >> 1) + (i >> 1) if i & 1 else i >> 1


@pytest.mark.parametrize("shape", [(16, 4, 6), (24, 6, 2), (8, 2, 2), (32, 10, 4)])
def test_rr4_model_matches_residual_restriction(shape):
    """k_cc_rr4: the coarse value is the mean of the residuals of the fine
    cells of the first colour (i + j + k even) among its 8 children; the
    kernel's thread forms coarse cells I0 .. I0+3 of a coarse row from
    4-wide vectors of the half-rows that hold those children, and writes
    them as two pairs (even and odd coarse cells)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(0)
    N = nx * ny * nz
    x, b, dg = rng.standard_normal(N), rng.standard_normal(N), rng.uniform(1, 2, N)
    bx = rng.uniform(0, 1, (nx + 1) * ny * nz)
    by = rng.uniform(0, 1, nx * (ny + 1) * nz)
    bz = rng.uniform(0, 1, nx * ny * (nz + 1))
    cix = lambda i, j, k: (k * ny + j) * nx + _split_pos(nx, i)

    def face(d, i, j, k):
        if d == 0: return (k * ny + j) * (nx + 1) + _split_pos(nx + 1, i)
        if d == 1: return (k * (ny + 1) + j) * nx + _split_pos(nx, i)
        return (k * ny + j) * nx + _split_pos(nx, i)
    gnx, gny, gnz = nx // 2, ny // 2, nz // 2
    ref = np.zeros(gnx * gny * gnz)
    for K, J, I in itertools.product(range(gnz), range(gny), range(gnx)):
        s = 0.0
        for o in range(8):
            if bin(o).count("1") & 1:
                continue
            i, j, k = 2 * I + (o & 1), 2 * J + ((o >> 1) & 1), 2 * K + ((o >> 2) & 1)
            c, off = cix(i, j, k), 0.0
            if i > 0: off += bx[face(0, i, j, k)] * x[cix(i - 1, j, k)]
            if i < nx - 1: off += bx[face(0, i + 1, j, k)] * x[cix(i + 1, j, k)]
            if j > 0: off += by[face(1, i, j, k)] * x[c - nx]
            if j < ny - 1: off += by[face(1, i, j + 1, k)] * x[c + nx]
            if k > 0: off += bz[face(2, i, j, k)] * x[c - nx * ny]
            if k < nz - 1: off += bz[face(2, i, j, k + 1)] * x[c + nx * ny]
            s += b[c] - (dg[c] * x[c] - off)
        ref[(K * gny + J) * gnx + _split_pos(gnx, I)] = s * 0.125
    out = np.full(gnx * gny * gnz, np.nan)
    hx, hf, sy, sz = nx >> 1, (nx + 2) >> 1, nx, nx * ny
    for K, J, I0 in itertools.product(range(gnz), range(gny), range(0, gnx, 4)):
        acc = [0.0] * 4
        for kk, jj in itertools.product(range(2), range(2)):
            j, k = 2 * J + jj, 2 * K + kk
            h = (j + k) & 1                       # the half holding the first colour's children
            rc = (k * ny + j) * nx
            c, o = rc + (hx if h else 0) + I0, rc + (0 if h else hx) + I0
            assert c % 4 == 0 and o % 4 == 0      # 16-byte vectors
            xc4, bb, d4, xo = x[c:c + 4], b[c:c + 4], dg[c:c + 4], x[o:o + 4]
            xb = (x[o + 4] if I0 + 4 < hx else 0.0) if h else (x[o - 1] if I0 > 0 else 0.0)
            xs = x[c - sy:c - sy + 4] if j > 0 else None
            xn = x[c + sy:c + sy + 4] if j < ny - 1 else None
            xd = x[c - sz:c - sz + 4] if k > 0 else None
            xu = x[c + sz:c + sz + 4] if k < nz - 1 else None
            fy0, fy1 = by[c + k * nx:c + k * nx + 4], by[c + k * nx + nx:c + k * nx + nx + 4]
            fz0, fz1 = bz[c:c + 4], bz[c + sz:c + sz + 4]
            rf = rc + k * ny + j
            for e in range(4):
                t = I0 + e
                i = 2 * t + h
                bxl, bxh = bx[rf + (hf + t if h else t)], bx[rf + (t + 1 if h else hf + t)]
                xw = xo[e] if h else (xo[e - 1] if e else xb)
                xe = (xo[e + 1] if e < 3 else xb) if h else xo[e]
                off = 0.0
                if i > 0: off += bxl * xw
                if i < nx - 1: off += bxh * xe
                if j > 0: off += fy0[e] * xs[e]
                if j < ny - 1: off += fy1[e] * xn[e]
                if k > 0: off += fz0[e] * xd[e]
                if k < nz - 1: off += fz1[e] * xu[e]
                acc[e] += bb[e] - (d4[e] * xc4[e] - off)
        hxc, row = gnx >> 1, (K * gny + J) * gnx
        out[row + (I0 >> 1)], out[row + (I0 >> 1) + 1] = acc[0] * 0.125, acc[2] * 0.125
        out[row + hxc + (I0 >> 1)], out[row + hxc + (I0 >> 1) + 1] = acc[1] * 0.125, acc[3] * 0.125
    assert not np.isnan(out).any()
    assert np.array_equal(out, ref)


# ---- k_cc_gs2_dot: the last colour pass with the fused sweep's partials ---
def _one_colour(g, b, dinv, x, bx, by, bz, col):
    x = x.copy()
    hf = (g.nx + 2) >> 1
    new = {}
    for k, j, i in itertools.product(range(g.nz), range(g.ny), range(g.nx)):
        if (i + j + k) & 1 != col:
            continue
        c, t, odd = cix(g, i, j, k), i >> 1, i & 1
        rf = (k * g.ny + j) * (g.nx + 1)
        s = 0.0
        if i > 0: s += bx[rf + (hf + t if odd else t)] * x[cix(g, i - 1, j, k)]
        if i < g.nx - 1: s += bx[rf + (t + 1 if odd else hf + t)] * x[cix(g, i + 1, j, k)]
        if j > 0: s += by[c + k * g.nx] * x[c - g.nx]
        if j < g.ny - 1: s += by[c + k * g.nx + g.nx] * x[c + g.nx]
        if k > 0: s += bz[c] * x[c - g.nx * g.ny]
        if k < g.nz - 1: s += bz[c + g.nx * g.ny] * x[c + g.nx * g.ny]
        new[c] = (b[c] + s) * dinv[c]
    for c, v in new.items():
        x[c] = v
    return x


def _gs2_dot(g, b, dinv, x, bx, by, bz, c1):
    """k_cc_gs2_dot: colour c1 by the fused sweep's threads (positions pq,
    pq + 1 of both halves of a tile row), with the b.x partial of every
    (plane, tile) over the same cells."""
    x = x.copy()
    hx, hf, sy, sz = g.nx >> 1, (g.nx + 2) >> 1, g.nx, g.nx * g.ny
    part, upd = {}, {}
    for k, ty_, tx_ in itertools.product(range(g.nz), range((g.ny + TY - 1) // TY), range((hx + HW - 1) // HW)):
        for tid in range(THREADS):
            j, pq = ty_ * TY + (tid >> 4), tx_ * HW + 2 * (tid & 15)
            if not (j < g.ny and pq < hx):
                continue
            h2 = (c1 + j + k) & 1
            rc = (k * g.ny + j) * g.nx
            c, o = rc + (hx if h2 else 0) + pq, rc + (0 if h2 else hx) + pq
            bb, bo, di, xo = b[c:c + 2], b[o:o + 2], dinv[c:c + 2], x[o:o + 2]
            xb = (x[o + 2] if pq + 2 < hx else 0.0) if h2 else (x[o - 1] if pq > 0 else 0.0)
            xs = x[c - sy:c - sy + 2] if j > 0 else [0, 0]
            xn = x[c + sy:c + sy + 2] if j < g.ny - 1 else [0, 0]
            xd = x[c - sz:c - sz + 2] if k > 0 else [0, 0]
            xu = x[c + sz:c + sz + 2] if k < g.nz - 1 else [0, 0]
            xw2 = [xo[0] if h2 else xb, xo[1] if h2 else xo[0]]
            xe2 = [xo[1] if h2 else xo[0], xb if h2 else xo[1]]
            rf = rc + k * g.ny + j
            s2 = [0.0, 0.0]
            for e in range(2):
                t = pq + e
                i = 2 * t + h2
                off = 0.0
                if i > 0: off += bx[rf + (hf + t if h2 else t)] * xw2[e]
                if i < g.nx - 1: off += bx[rf + (t + 1 if h2 else hf + t)] * xe2[e]
                if j > 0: off += by[c + k * g.nx + e] * xs[e]
                if j < g.ny - 1: off += by[c + k * g.nx + g.nx + e] * xn[e]
                if k > 0: off += bz[c + e] * xd[e]
                if k < g.nz - 1: off += bz[c + sz + e] * xu[e]
                s2[e] = (bb[e] + off) * di[e]
            upd[c], upd[c + 1] = s2
            b0, b1 = (bo, bb) if h2 else (bb, bo)
            v0, v1 = (xo, s2) if h2 else (s2, xo)
            key = (k, ty_, tx_)
            part[key] = part.get(key, 0.0) + b0[0] * v0[0] + b0[1] * v0[1] + b1[0] * v1[0] + b1[1] * v1[1]
    for c, v in upd.items():
        x[c] = v
    return x, part


@pytest.mark.parametrize("shape", [(16, 5, 3), (80, 20, 4), (48, 18, 7)])
def test_gs2_dot_model_matches_fused_partials(shape):
    """The colour passes end with k_cc_gs2_dot, which forms the same (plane,
    tile) partials of b.x over the same cells as the fused sweep with r.z."""
    g = Grid(*shape)
    rng = np.random.default_rng(3)
    n = g.nx * g.ny * g.nz
    b, dinv, x = rng.standard_normal(n), rng.uniform(0.1, 0.3, n), rng.standard_normal(n)
    bx = rng.uniform(0, 1, (g.nx + 1) * g.ny * g.nz)
    by = rng.uniform(0, 1, g.nx * (g.ny + 1) * g.nz)
    bz = rng.uniform(0, 1, g.nx * g.ny * (g.nz + 1))
    for c0 in (0, 1):
        ref = colour_passes(g, b, dinv, x, bx, by, bz, c0, False)
        out, part = _gs2_dot(g, b, dinv, _one_colour(g, b, dinv, x, bx, by, bz, c0), bx, by, bz, 1 - c0)
        assert np.abs(out - ref).max() <= 1e-12 * np.abs(ref).max()
        _, fused_part = fused_sweep(g, b, dinv, x, bx, by, bz, c0, 3)
        assert set(part) == set(fused_part)
        assert max(abs(part[key] - fused_part[key]) for key in part) <= 1e-12
