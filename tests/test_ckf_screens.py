"""Soundness of the track-finding navigation's FP32 screens (host model, no GPU).

The navigation decides, in FP64, which layers a straight line reaches ahead and which modules a
parabola crosses (Sec. 2, track finding over the detector's layers). The kernels first evaluate
each test in FP32 and skip the FP64 evaluation only where an error bound shows that it would
reject too. This file restates each FP32 screen as the kernel evaluates it (numpy float32
operations, every one rounded; the kernel's compiler may fuse a product and a sum, which rounds
less) and checks, on lines and parabolas aimed at the decision edges, that a screen never skips
what the FP64 test accepts. The FP64 tests are written out from their definitions in the
track-finding interface: a disk face reached within its radial extent, a barrel face reached
from inside within its z extent, a module crossed ahead within its half extents plus the helix
margin."""

import numpy as np

F32, F64 = np.float32, np.float64
RNG = np.random.default_rng(20261204)
N = 200_000


def f32(x):
    return np.asarray(x, dtype=F64).astype(F32)


def fma32(a, b, c):
    # a b is exact in FP64 for FP32 operands; one rounding of the sum to FP32 (up to a tie
    # broken twice, within the screens' bounds either way)
    return (a.astype(F64) * b.astype(F64) + c.astype(F64)).astype(F32)


def unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def random_dirs(n):
    return unit(RNG.normal(size=(n, 3)))


# ---------------------------------------------------------------------------------------------
# disk face: radial extent


def disk_fp64(x, T, zface, lo, hi):
    """-1 (not reached within the extent) as the FP64 test decides, else the path."""
    dz = zface - x[:, 2]
    ahead = ((dz > 0) & (T[:, 2] > 0)) | ((dz < 0) & (T[:, 2] < 0))
    with np.errstate(divide="ignore", invalid="ignore"):
        s = dz / T[:, 2]
        r = np.hypot(x[:, 0] + s * T[:, 0], x[:, 1] + s * T[:, 1])
    ok = ahead & (s > 0) & ~((r < lo) | (r > hi))
    return ok


def disk_screen(x, T, zface, lo, hi):
    """True where the FP32 screen returns -1 (the kernel's disk branch, after the sign test)."""
    xf, Tf = f32(x), f32(T)
    dz = zface - x[:, 2]
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        sf = f32(dz) / Tf[:, 2]
        px, py = fma32(sf, Tf[:, 0], xf[:, 0]), fma32(sf, Tf[:, 1], xf[:, 1])
        rq = np.sqrt(px * px + py * py)
        e = F32(1e-6) * (np.abs(xf[:, 0]) + np.abs(xf[:, 1]) + np.abs(sf) * (np.abs(Tf[:, 0]) + np.abs(Tf[:, 1])) + rq) \
            + F32(1e-3)
        return (rq + e < f32(lo)) | (rq - e > f32(hi))


def test_disk_radial_screen_never_skips_a_reached_face():
    skips = 0
    for zface in (601.0, -1401.0, 3001.0):
        r_inner, n_rings, pitch = 32.0, 15, 68.0
        lo, hi = r_inner - 10.0, r_inner + n_rings * pitch + 10.0
        edge = np.where(RNG.random(N) < 0.5, lo, hi)
        rho = edge + RNG.uniform(-0.01, 0.01, N) * 10.0 ** RNG.integers(-3, 2, N)
        phi = RNG.uniform(0, 2 * np.pi, N)
        P = np.stack([rho * np.cos(phi), rho * np.sin(phi), np.full(N, zface)], axis=1)
        # starts anywhere in the tracker on the near side of the face
        zs = zface - np.sign(zface) * RNG.uniform(1.0, 2500.0, N)
        rs, ps = RNG.uniform(0.0, 1100.0, N), RNG.uniform(0, 2 * np.pi, N)
        x = np.stack([rs * np.cos(ps), rs * np.sin(ps), zs], axis=1)
        T = unit(P - x)
        skip = disk_screen(x, T, zface, lo, hi)
        reached = disk_fp64(x, T, zface, lo, hi)
        assert not np.any(skip & reached), "the disk screen skipped a face the FP64 test reaches"
        skips += int(skip.sum())
    assert skips > 0.08 * 3 * N  # outside the error band it decides (about 16 % of these samples)


# ---------------------------------------------------------------------------------------------
# barrel face: the point outside it, and the z extent


def barrel_fp64(x, T, rf, zmax):
    aa = T[:, 0] ** 2 + T[:, 1] ** 2
    b = x[:, 0] * T[:, 0] + x[:, 1] * T[:, 1]
    c = x[:, 0] ** 2 + x[:, 1] ** 2 - rf * rf
    inside = (aa > 0) & (c < 0)
    with np.errstate(divide="ignore", invalid="ignore"):
        s = (-b + np.sqrt(b * b - aa * c)) / aa
        ok = inside & ~(np.abs(x[:, 2] + s * T[:, 2]) > zmax) & (s > 0)
    return ok


def barrel_screen(x, T, rf, zmax):
    """True where one of the kernel's two barrel screens returns -1."""
    xf, Tf = f32(x), f32(T)
    rff, zmf = f32(rf), f32(zmax)
    p2f = xf[:, 0] * xf[:, 0] + xf[:, 1] * xf[:, 1]
    f2f = rff * rff
    outside = p2f - f2f > F32(1e-6) * (p2f + f2f)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        tz = Tf[:, 2]
        zl = np.copysign(zmf + F32(1e-3) + F32(1e-6) * np.abs(xf[:, 2]), tz).astype(F32)
        dzf = zl - xf[:, 2]
        beyond = np.where(tz > 0, dzf <= 0, dzf >= 0)
        szf = dzf / tz
        tp = np.abs(Tf[:, 0]) + np.abs(Tf[:, 1])
        px, py = fma32(szf, Tf[:, 0], xf[:, 0]), fma32(szf, Tf[:, 1], xf[:, 1])
        rq = np.sqrt(px * px + py * py)
        e = F32(1e-6) * (np.abs(xf[:, 0]) + np.abs(xf[:, 1]) + szf * tp + rq +
                         (np.abs(zl) + np.abs(xf[:, 2])) * tp / np.abs(tz)) + F32(1e-3)
        short = rq + e < rff
    zscreen = (tz != 0) & (beyond | short)
    return outside | zscreen, outside


def test_barrel_screens_never_skip_a_reached_face():
    skips_out = skips_z = 0
    zmax = 0.5 * 18 * 68.0 + 10.0
    for r in (32.0, 150.0, 1000.0):
        rf = np.sqrt((r + 1.0) ** 2 + 15.0 ** 2)
        # (a) starts near the face radius, both sides: the point-outside screen
        rho = rf * (1.0 + RNG.uniform(-1e-5, 1e-5, N) * 10.0 ** RNG.integers(-2, 3, N))
        ps = RNG.uniform(0, 2 * np.pi, N)
        x = np.stack([rho * np.cos(ps), rho * np.sin(ps), RNG.uniform(-3000, 3000, N)], axis=1)
        T = random_dirs(N)
        skip, outside = barrel_screen(x, T, rf, zmax)
        assert not np.any(skip & barrel_fp64(x, T, rf, zmax)), "a barrel screen skipped a reached face"
        skips_out += int(outside.sum())
        # (b) lines from inside that meet the face near z = +-zmax: the z-extent screen
        zt = np.where(RNG.random(N) < 0.5, 1.0, -1.0) * (zmax + RNG.uniform(-0.01, 0.01, N) *
                                                         10.0 ** RNG.integers(-3, 2, N))
        pt = RNG.uniform(0, 2 * np.pi, N)
        P = np.stack([rf * np.cos(pt), rf * np.sin(pt), zt], axis=1)
        ri, pi_ = rf * np.sqrt(RNG.uniform(0.0, 0.999, N)), RNG.uniform(0, 2 * np.pi, N)
        x = np.stack([ri * np.cos(pi_), ri * np.sin(pi_), RNG.uniform(-3000, 3000, N)], axis=1)
        T = unit(P - x)
        skip, outside = barrel_screen(x, T, rf, zmax)
        assert not np.any(skip & barrel_fp64(x, T, rf, zmax)), "the z-extent screen skipped a reached face"
        skips_z += int((skip & ~outside).sum())
    assert skips_out > 0.14 * 3 * N and skips_z > 0.02 * 3 * N  # about 29 % and 4 % of these samples


# ---------------------------------------------------------------------------------------------
# module crossing: the parabola x + s T + s^2/2 k against the module's bounds plus margin


def crossing_fp64(x, T, k, bend, c, u, v, n, hu, hv):
    """True where the FP64 test accepts the module (crossed ahead within bounds and margin)."""
    d = c - x
    dist, an, bn = (n * d).sum(1), (n * T).sum(1), (n * k).sum(1)
    with np.errstate(divide="ignore", invalid="ignore"):
        disc = an * an + 2.0 * bn * dist
        q2 = 2.0 * dist / (an + np.copysign(np.sqrt(np.maximum(disc, 0.0)), an))
        s = np.where((disc >= 0) & np.isfinite(q2), q2, dist / an)
        h = 0.5 * s * s
        q = x + s[:, None] * T + h[:, None] * k - c
        margin = 1.0 + s ** 3 * bend ** 2 / 6.0
        ok = (an != 0) & (s > 1e-3) & ~((np.abs((u * q).sum(1)) > hu + margin) | (np.abs((v * q).sum(1)) > hv + margin))
    return ok


def crossing_screen(x, T, k, bend, c, u, v, n, hu, hv):
    """True where the kernel's FP32 screen (`surely_outside`) skips the module."""
    def dot(a, b):
        return a[:, 0] * b[:, 0] + a[:, 1] * b[:, 1] + a[:, 2] * b[:, 2]
    xf, Tf, kf = f32(x), f32(T), f32(k)
    uf, vf, nf, cf = f32(u), f32(v), f32(n), f32(c)
    knorm = np.abs(kf).sum(1, dtype=F32) * F32(1.00001)
    bendf = f32(bend) * F32(1.00001)
    xn = np.abs(xf).sum(1, dtype=F32)
    df = cf - xf
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        an = dot(nf, Tf)
        dist, bn = dot(nf, df), dot(nf, kf)
        disc = an * an + F32(2) * bn * dist
        sf = F32(2) * dist / (an + np.copysign(np.sqrt(disc), an).astype(F32))
        valid = (np.abs(an) > F32(0.05)) & (disc > F32(0.25) * an * an) & np.isfinite(sf)
        as_, h = np.abs(sf), F32(0.5) * sf * sf
        q = -df + sf[:, None] * Tf + h[:, None] * kf
        dn, qn = np.abs(df).sum(1, dtype=F32), np.abs(q).sum(1, dtype=F32)
        ecx = F32(1.2e-7) * (np.abs(cf).sum(1, dtype=F32) + xn)
        rs = F32(1e-5) + F32(2e-6) * np.abs(bn) * dn / (an * an)
        ds = rs * as_ + (F32(1e-5) * dn + F32(2.5) * ecx) / np.abs(an)
        err = F32(1e-3) + ecx + ds * (F32(1) + (as_ + ds) * knorm) + F32(1e-6) * (dn + qn)
        sup = (as_ + ds) * F32(1.00001)
        margin = (F32(1) + sup * sup * sup * bendf * bendf / F32(6)) * F32(1.00001)
        out = (np.abs(dot(uf, q)) - err > f32(hu) + margin) | (np.abs(dot(vf, q)) - err > f32(hv) + margin)
    return valid & out


def test_module_crossing_screen_never_skips_a_crossed_module():
    hu, hv = 15.0, 35.0
    skips = 0
    for far in (False, False, True):
        # modules anywhere in the tracker, frames at random orientations; last, modules far from
        # the origin reached on short paths, where the rounding of the FP32 centre and position
        # copies is most of the error
        zc = np.where(RNG.random(N) < 0.5, 1.0, -1.0) * RNG.uniform(2500, 3000, N) if far else RNG.uniform(-3000, 3000, N)
        c = np.stack([RNG.uniform(-1000, 1000, N), RNG.uniform(-1000, 1000, N), zc], axis=1)
        n = random_dirs(N)
        u = unit(np.cross(n, random_dirs(N)))
        v = np.cross(n, u)
        # a parabola that meets the plane at path s0 near the edge of the bounds plus margin
        s0 = 10.0 ** RNG.uniform(-1.0, 0.7, N) if far else RNG.uniform(2.0, 600.0, N)
        kmag = RNG.uniform(0.0, 6e-3, N)
        bend = kmag / RNG.uniform(0.3, 1.0, N)
        margin = 1.0 + s0 ** 3 * bend ** 2 / 6.0
        side = np.where(RNG.random(N) < 0.5, 1.0, -1.0)
        delta = RNG.uniform(-0.05, 0.05, N) * 10.0 ** RNG.integers(-3, 2, N)
        along_u = RNG.random(N) < 0.5
        a = np.where(along_u, side * (hu + margin + delta), RNG.uniform(-hu, hu, N))
        b = np.where(along_u, RNG.uniform(-hv, hv, N), side * (hv + margin + delta))
        P = c + a[:, None] * u + b[:, None] * v
        # direction with |n.T| from grazing to normal, curvature perpendicular to it
        an = np.where(RNG.random(N) < 0.5, 1.0, -1.0) * RNG.uniform(0.02, 1.0, N)
        w = unit(np.cross(n, random_dirs(N)))
        T = an[:, None] * n + np.sqrt(1.0 - an ** 2)[:, None] * w
        k = kmag[:, None] * unit(np.cross(T, random_dirs(N)))
        x = P - s0[:, None] * T - (0.5 * s0 ** 2)[:, None] * k
        skip = crossing_screen(x, T, k, bend, c, u, v, n, hu, hv)
        crossed = crossing_fp64(x, T, k, bend, c, u, v, n, hu, hv)
        assert not np.any(skip & crossed), "the crossing screen skipped a module the FP64 test accepts"
        skips += int(skip.sum())
    assert skips > 0.10 * 3 * N  # about 20 % of these samples
