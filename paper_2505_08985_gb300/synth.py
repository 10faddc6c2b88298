"""Seeded synthetic workloads: normal maps, P-NDF queries and light directions.

This module only manufactures inputs.  It holds none of the P-NDF or
projected-area arithmetic; both the CUDA path and the FP64 oracle consume what
it returns.  The paper's own normal maps (three 1024^2 maps, Sec. 5; a flake
map, App. D) and scenes are not available, so every map here is a procedural
stand-in with the structure the paper describes: smooth bumps (isotropic),
V-groove scratches over value noise, and Voronoi metallic flakes.

Conventions
-----------
* A normal map ``st`` is a ``(N, N, 2)`` tensor indexed ``st[j, i]`` for the
  texel at integer coordinate ``u = (i, j)`` (``i`` along x / columns, ``j``
  along y / rows).  The two channels are the projected-hemisphere normal
  ``n = (s, t)`` (Sec. 3, Eq. 2: only the xy part of the unit normal).
* Heights are in texel units; normals come from central differences of the
  height (one-sided at the border) and are clamped component-wise to
  ``|s|, |t| <= 0.4``.
* A query is 8 floats ``(x, y, sxx, sxy, syy, ms, mt, 0)``: footprint centre in
  texel coordinates, the 2x2 footprint covariance (texel^2) and the query
  normal.

All random draws for per-feature parameters (bump centres, groove endpoints,
cell seeds, query parameters) come from a CPU ``torch.Generator`` seeded with
the workload seed; per-texel white noise is drawn on the target device from a
generator with the same seed.  Generation on CPU is therefore reproducible
across machines; large maps are generated on the GPU for speed.
"""

from __future__ import annotations

import math
from dataclasses import dataclass

import torch

CLAMP = 0.4


def _cpu_gen(seed: int, stream: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed((int(seed) * 1_000_003 + int(stream) * 7919) & 0x7FFF_FFFF_FFFF)
    return g


def _dev_gen(seed: int, stream: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((int(seed) * 1_000_033 + int(stream) * 104_729) & 0x7FFF_FFFF_FFFF)
    return g


def _u(g, n, lo, hi, dtype=torch.float64):
    return lo + (hi - lo) * torch.rand(n, generator=g, dtype=dtype)


def _log_u(g, n, lo, hi):
    return torch.exp(_u(g, n, math.log(lo), math.log(hi)))


# ---------------------------------------------------------------------------
# height fields and normal maps
# ---------------------------------------------------------------------------

def normals_from_height(h: torch.Tensor, clamp: float = CLAMP) -> torch.Tensor:
    """(N, N) height -> (N, N, 2) float32 projected normals (s, t).

    The unit normal of z = h(x, y) is (-h_x, -h_y, 1) / sqrt(1 + h_x^2 + h_y^2);
    (s, t) is its xy part, clamped to |s|, |t| <= clamp.
    """
    h = h.to(torch.float64) if h.device.type == "cpu" else h.to(torch.float32)
    hx = torch.empty_like(h)
    hy = torch.empty_like(h)
    hx[:, 1:-1] = 0.5 * (h[:, 2:] - h[:, :-2])
    hx[:, 0] = h[:, 1] - h[:, 0]
    hx[:, -1] = h[:, -1] - h[:, -2]
    hy[1:-1, :] = 0.5 * (h[2:, :] - h[:-2, :])
    hy[0, :] = h[1, :] - h[0, :]
    hy[-1, :] = h[-1, :] - h[-2, :]
    inv = torch.rsqrt(1.0 + hx * hx + hy * hy)
    st = torch.stack((-hx * inv, -hy * inv), dim=-1)
    return st.clamp_(-clamp, clamp).to(torch.float32).contiguous()


def bumps_height(n: int, n_bumps: int, seed: int, device="cpu",
                 amp=(0.5, 2.0), sig=(2.0, 16.0), noise=0.05) -> torch.Tensor:
    """Sum of Gaussian bumps (amplitude U(amp), width U(sig), centre U[0,N)^2)
    plus N(0, noise^2) white noise, in texel units."""
    g = _cpu_gen(seed, 1)
    cx = _u(g, n_bumps, 0.0, n)
    cy = _u(g, n_bumps, 0.0, n)
    a = _u(g, n_bumps, *amp)
    s = _u(g, n_bumps, *sig)
    dt = torch.float64 if torch.device(device).type == "cpu" else torch.float32
    h = torch.zeros(n, n, dtype=dt, device=device)
    ax = torch.arange(n, dtype=dt, device=device)
    for k in range(n_bumps):
        r = float(4.5 * s[k])
        i0, i1 = max(0, int(cx[k] - r)), min(n, int(cx[k] + r) + 2)
        j0, j1 = max(0, int(cy[k] - r)), min(n, int(cy[k] + r) + 2)
        if i0 >= i1 or j0 >= j1:
            continue
        gx = torch.exp(-0.5 * ((ax[i0:i1] - float(cx[k])) / float(s[k])) ** 2)
        gy = torch.exp(-0.5 * ((ax[j0:j1] - float(cy[k])) / float(s[k])) ** 2)
        h[j0:j1, i0:i1] += float(a[k]) * gy[:, None] * gx[None, :]
    if noise > 0:
        h += noise * torch.randn(n, n, generator=_dev_gen(seed, 2, device), dtype=dt, device=device)
    return h


def value_noise(n: int, seed: int, device="cpu", base_period=64, amplitude=1.0, octaves=3) -> torch.Tensor:
    """Lattice value noise with smoothstep interpolation, summed over octaves
    (period halves and amplitude halves per octave)."""
    dt = torch.float64 if torch.device(device).type == "cpu" else torch.float32
    h = torch.zeros(n, n, dtype=dt, device=device)
    ax = torch.arange(n, dtype=dt, device=device)
    period, amp = float(base_period), float(amplitude)
    for o in range(octaves):
        cells = int(math.ceil(n / period)) + 2
        lat = (2.0 * torch.rand(cells, cells, generator=_cpu_gen(seed, 10 + o), dtype=torch.float64) - 1.0)
        lat = lat.to(device=device, dtype=dt) * amp
        f = ax / period
        i0 = torch.floor(f).long()
        fr = f - i0.to(dt)
        w = fr * fr * (3.0 - 2.0 * fr)
        # rows: y, cols: x
        v00 = lat[i0[:, None], i0[None, :]]
        v01 = lat[i0[:, None], i0[None, :] + 1]
        v10 = lat[i0[:, None] + 1, i0[None, :]]
        v11 = lat[i0[:, None] + 1, i0[None, :] + 1]
        wx = w[None, :]
        wy = w[:, None]
        h += (v00 * (1 - wx) + v01 * wx) * (1 - wy) + (v10 * (1 - wx) + v11 * wx) * wy
        period *= 0.5
        amp *= 0.5
    return h


def carve_grooves(h: torch.Tensor, n_grooves: int, seed: int,
                  length=(32.0, 512.0), half_width=(0.5, 2.0), depth=(0.2, 1.0)) -> torch.Tensor:
    """Subtract V-groove profiles depth * max(0, 1 - dist/half_width) along
    random line segments (start U[0,N)^2, direction U(0, 2pi), length U(length))."""
    n = h.shape[0]
    g = _cpu_gen(seed, 20)
    x0 = _u(g, n_grooves, 0.0, n)
    y0 = _u(g, n_grooves, 0.0, n)
    th = _u(g, n_grooves, 0.0, 2 * math.pi)
    ln = _u(g, n_grooves, *length)
    hw = _u(g, n_grooves, *half_width)
    dp = _u(g, n_grooves, *depth)
    dt = h.dtype
    dev = h.device
    for k in range(n_grooves):
        ax, ay = float(x0[k]), float(y0[k])
        bx, by = ax + float(ln[k]) * math.cos(float(th[k])), ay + float(ln[k]) * math.sin(float(th[k]))
        w = float(hw[k])
        i0, i1 = max(0, int(math.floor(min(ax, bx) - w)) - 1), min(n, int(math.ceil(max(ax, bx) + w)) + 2)
        j0, j1 = max(0, int(math.floor(min(ay, by) - w)) - 1), min(n, int(math.ceil(max(ay, by) + w)) + 2)
        if i0 >= i1 or j0 >= j1:
            continue
        px = torch.arange(i0, i1, dtype=dt, device=dev)[None, :]
        py = torch.arange(j0, j1, dtype=dt, device=dev)[:, None]
        vx, vy = bx - ax, by - ay
        L2 = vx * vx + vy * vy
        t = (((px - ax) * vx + (py - ay) * vy) / L2).clamp(0.0, 1.0)
        dx = px - (ax + t * vx)
        dy = py - (ay + t * vy)
        dist = torch.sqrt(dx * dx + dy * dy)
        h[j0:j1, i0:i1] -= float(dp[k]) * torch.clamp(1.0 - dist / w, min=0.0)
    return h


def flake_normals(n: int, n_cells: int, seed: int, device="cpu",
                  cell_sigma=0.15, texel_noise=0.005, chunk_rows=1024) -> torch.Tensor:
    """Voronoi metallic flakes: jittered-grid seeds (one per grid cell, about
    n_cells in total), each cell with a constant normal ~ N(0, cell_sigma^2 I),
    plus N(0, texel_noise^2) per texel.  Nearest seed is searched among the
    3x3 neighbouring grid cells.  Returns (N, N, 2) float32, clamped."""
    gcount = max(1, int(round(math.sqrt(n_cells))))
    cell = n / gcount
    g = _cpu_gen(seed, 30)
    jx = torch.rand(gcount, gcount, generator=g, dtype=torch.float64)
    jy = torch.rand(gcount, gcount, generator=g, dtype=torch.float64)
    cn = cell_sigma * torch.randn(gcount, gcount, 2, generator=g, dtype=torch.float64)
    dt = torch.float64 if torch.device(device).type == "cpu" else torch.float32
    # seed positions, padded by one ring (clamped copies never win past the border ring)
    sx = ((torch.arange(gcount, dtype=torch.float64)[None, :] + jx) * cell).to(device=device, dtype=dt)
    sy = ((torch.arange(gcount, dtype=torch.float64)[:, None] + jy) * cell).to(device=device, dtype=dt)
    cn = cn.to(device=device, dtype=dt)
    out = torch.empty(n, n, 2, dtype=torch.float32, device=device)
    px = torch.arange(n, dtype=dt, device=device)
    gxi = torch.clamp((px / cell).long(), 0, gcount - 1)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        py = torch.arange(r0, r1, dtype=dt, device=device)
        gyi = torch.clamp((py / cell).long(), 0, gcount - 1)
        best = torch.full((r1 - r0, n), float("inf"), dtype=dt, device=device)
        bi = torch.zeros((r1 - r0, n), dtype=torch.long, device=device)
        bj = torch.zeros((r1 - r0, n), dtype=torch.long, device=device)
        for oy in (-1, 0, 1):
            cj = torch.clamp(gyi + oy, 0, gcount - 1)[:, None].expand(r1 - r0, n)
            for ox in (-1, 0, 1):
                ci = torch.clamp(gxi + ox, 0, gcount - 1)[None, :].expand(r1 - r0, n)
                dx = px[None, :] - sx[cj, ci]
                dy = py[:, None] - sy[cj, ci]
                d2 = dx * dx + dy * dy
                better = d2 < best
                best = torch.where(better, d2, best)
                bi = torch.where(better, ci, bi)
                bj = torch.where(better, cj, bj)
        out[r0:r1] = cn[bj, bi].to(torch.float32)
    if texel_noise > 0:
        out += texel_noise * torch.randn(n, n, 2, generator=_dev_gen(seed, 31, device),
                                         dtype=torch.float32, device=device)
    return out.clamp_(-CLAMP, CLAMP).contiguous()


def affine_normals(n: int, n0, M) -> torch.Tensor:
    """n(u) = n0 + M u on the integer grid (exact when n0, M are dyadic)."""
    n0 = torch.as_tensor(n0, dtype=torch.float64)
    M = torch.as_tensor(M, dtype=torch.float64)
    ax = torch.arange(n, dtype=torch.float64)
    ii = ax[None, :].expand(n, n)
    jj = ax[:, None].expand(n, n)
    s = n0[0] + M[0, 0] * ii + M[0, 1] * jj
    t = n0[1] + M[1, 0] * ii + M[1, 1] * jj
    return torch.stack((s, t), dim=-1).to(torch.float32).contiguous()


# ---------------------------------------------------------------------------
# workload maps
# ---------------------------------------------------------------------------

def bumps_map(n=256, n_bumps=64, seed=1, device="cpu") -> torch.Tensor:
    return normals_from_height(bumps_height(n, n_bumps, seed, device))


def scratch_map(n=2048, n_grooves=2000, seed=2, device="cpu") -> torch.Tensor:
    h = value_noise(n, seed, device)
    h = carve_grooves(h, n_grooves, seed)
    return normals_from_height(h)


def flake_map(n=8192, n_cells=200_000, seed=3, device="cpu") -> torch.Tensor:
    return flake_normals(n, n_cells, seed, device)


def mixed_map(n=16384, n_cells=800_000, n_grooves=8000, seed=5, device="cpu") -> torch.Tensor:
    """Scratches over flakes: groove/noise slopes added to the flake normals,
    then clamped (the stand-in for the combined map)."""
    h = value_noise(n, seed, device)
    h = carve_grooves(h, n_grooves, seed)
    st = normals_from_height(h, clamp=10.0)
    st += flake_normals(n, n_cells, seed, device)
    return st.clamp_(-CLAMP, CLAMP).contiguous()


# ---------------------------------------------------------------------------
# queries
# ---------------------------------------------------------------------------

@dataclass
class QueryMix:
    sigma: tuple = (4.0, 4.0)       # major sigma range (log-uniform); equal ends = fixed
    aspect: tuple = (1.0, 1.0)      # major/minor ratio, uniform
    frac_near: float = 1.0          # fraction of query normals drawn near the footprint's normals
    near_noise: float = 0.02        # N(0, near_noise^2) added to the sampled texel normal
    centre_margin: float = 0.0      # centres uniform in [margin, N-1-margin]^2


def make_queries(st: torch.Tensor, nq: int, mix: QueryMix, seed: int) -> torch.Tensor:
    """(nq, 8) float32 queries on st's device.  Random texel inside the
    footprint: u = x + chol(Sigma) z with z ~ N(0, I) clipped to |z| <= 4,
    rounded to the nearest texel and clamped into the map."""
    n = st.shape[0]
    dev = st.device
    g = _cpu_gen(seed, 40)
    lo, hi = mix.centre_margin, (n - 1) - mix.centre_margin
    x = _u(g, nq, lo, hi)
    y = _u(g, nq, lo, hi)
    if mix.sigma[0] == mix.sigma[1]:
        s1 = torch.full((nq,), float(mix.sigma[0]), dtype=torch.float64)
    else:
        s1 = _log_u(g, nq, *mix.sigma)
    asp = _u(g, nq, *mix.aspect) if mix.aspect[0] != mix.aspect[1] else torch.full((nq,), float(mix.aspect[0]), dtype=torch.float64)
    s2 = s1 / asp
    th = _u(g, nq, 0.0, math.pi)
    c, s = torch.cos(th), torch.sin(th)
    sxx = c * c * s1 * s1 + s * s * s2 * s2
    syy = s * s * s1 * s1 + c * c * s2 * s2
    sxy = c * s * (s1 * s1 - s2 * s2)
    # covariance rounded to float32 first, so both consumers see the same SPD matrix
    sxx32, sxy32, syy32 = sxx.float().double(), sxy.float().double(), syy.float().double()
    # pick a texel from the footprint Gaussian
    z = torch.randn(nq, 2, generator=g, dtype=torch.float64)
    zn = torch.linalg.vector_norm(z, dim=1, keepdim=True).clamp(min=1e-30)
    z = torch.where(zn > 4.0, z * (4.0 / zn), z)
    l11 = torch.sqrt(sxx32)
    l21 = sxy32 / l11
    l22 = torch.sqrt(torch.clamp(syy32 - l21 * l21, min=0.0))
    ux = x + l11 * z[:, 0]
    uy = y + l21 * z[:, 0] + l22 * z[:, 1]
    ti = torch.clamp(torch.round(ux), 0, n - 1).long()
    tj = torch.clamp(torch.round(uy), 0, n - 1).long()
    near = st[tj.to(dev), ti.to(dev)].to("cpu", torch.float64)
    near = near + mix.near_noise * torch.randn(nq, 2, generator=g, dtype=torch.float64)
    unif = _u(g, (nq, 2), -CLAMP, CLAMP)
    pick = (torch.rand(nq, generator=g, dtype=torch.float64) < mix.frac_near)[:, None]
    m = torch.where(pick, near, unif)
    q = torch.stack((x, y, sxx32, sxy32, syy32, m[:, 0], m[:, 1], torch.zeros(nq, dtype=torch.float64)), dim=1)
    return q.to(torch.float32).to(dev).contiguous()


def hemisphere_dirs(nq: int, seed: int, device="cpu", min_z=1e-3) -> torch.Tensor:
    """(nq, 3) float32 unit directions uniform on the upper hemisphere (z >= min_z)."""
    g = _cpu_gen(seed, 50)
    z = _u(g, nq, min_z, 1.0)
    phi = _u(g, nq, 0.0, 2 * math.pi)
    r = torch.sqrt(torch.clamp(1 - z * z, min=0.0))
    w = torch.stack((r * torch.cos(phi), r * torch.sin(phi), z), dim=1)
    return w.to(torch.float32).to(device).contiguous()


# workload recipes named by what they are -----------------------------------

BUMPS_256 = dict(n=256, queries=4096, mix=QueryMix(sigma=(4.0, 4.0)), seed=1)
SCRATCH_2048 = dict(n=2048, queries=1 << 20, mix=QueryMix(sigma=(1.0, 64.0), aspect=(1.0, 4.0), frac_near=0.7), seed=2)
FLAKE_8192 = dict(n=8192, queries=1 << 22, mix=QueryMix(sigma=(1.0, 512.0), frac_near=0.7), seed=3)
MIXED_16384 = dict(n=16384, queries=1 << 23, mix=QueryMix(sigma=(1.0, 1024.0), frac_near=0.7), seed=5)


# ---------------------------------------------------------------------------
# camera-driven queries (serving workload)
# ---------------------------------------------------------------------------

def camera_queries(n_map: int, nq: int, seed: int, tilt_deg=(0.0, 75.0), dist=(0.3, 3.0), fov_deg=40.0,
                   image=1024, device="cpu") -> torch.Tensor:
    """(nq, 8) float32 CPU queries seen by a seeded pinhole camera over the
    textured plane z = 0 (the map spans the world square [0, 1]^2, texel units
    = world * n_map).

    The camera looks at a random point of the map from distance log-U(dist)
    with tilt U(tilt_deg) from the plane's normal; nq random pixels of an
    image x image view are traced.  A pixel's footprint covariance is
    Sigma = J J^T with J the exact ray differentials of the plane hit point
    (texels per pixel), scaled down where needed so 4 sigma <= n_map / 2.  The
    query normal is the xy part of the half vector between a random light
    direction (uniform on the upper hemisphere) and the view direction.
    Per-pixel draws come from a generator on `device` (the camera itself from
    a CPU generator), so large batches can be made on the GPU.
    """
    g = _cpu_gen(seed, 60)
    tilt = math.radians(float(_u(g, 1, *tilt_deg)))
    yaw = float(_u(g, 1, 0.0, 2 * math.pi))
    d0 = float(_log_u(g, 1, *dist))
    target = torch.stack([_u(g, 1, 0.2, 0.8), _u(g, 1, 0.2, 0.8), torch.zeros(1, dtype=torch.float64)]).squeeze(1)
    back = torch.tensor([math.sin(tilt) * math.cos(yaw), math.sin(tilt) * math.sin(yaw), math.cos(tilt)],
                        dtype=torch.float64)
    cam = target + d0 * back
    fwd = -back
    up0 = torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64) if abs(math.cos(tilt)) < 0.999 else \
        torch.tensor([math.cos(yaw), math.sin(yaw), 0.0], dtype=torch.float64)
    right = torch.linalg.cross(fwd, up0)
    right = right / torch.linalg.vector_norm(right)
    up = torch.linalg.cross(right, fwd)
    half = math.tan(math.radians(fov_deg) / 2)
    px = 2.0 * half / image  # image-plane step per pixel at unit distance
    dev = torch.device(device)
    gd = _dev_gen(seed, 61, dev)
    cam, fwd, right, up = (v.to(dev) for v in (cam, fwd, right, up))

    def ud(n, lo, hi):
        return lo + (hi - lo) * torch.rand(n, generator=gd, dtype=torch.float64, device=dev)

    out = []
    need = nq
    while need > 0:
        m = int(need * 1.3) + 16
        a = ud(m, -half, half)
        b = ud(m, -half, half)
        d = fwd[None] + a[:, None] * right[None] + b[:, None] * up[None]
        ok = d[:, 2] < -1e-6
        a, b, d = a[ok], b[ok], d[ok]
        t = -cam[2] / d[:, 2]
        hit = cam[None] + t[:, None] * d
        # exact differentials of the plane hit point w.r.t. one pixel step
        J = []
        for axis in (right, up):
            dd = px * axis
            dt = -t * dd[2] / d[:, 2]
            J.append((t[:, None] * dd[None, :2] + dt[:, None] * d[:, :2]) * n_map)
        Ja, Jb = J  # columns of J (texels per pixel)
        sxx = Ja[:, 0] ** 2 + Jb[:, 0] ** 2
        syy = Ja[:, 1] ** 2 + Jb[:, 1] ** 2
        sxy = Ja[:, 0] * Ja[:, 1] + Jb[:, 0] * Jb[:, 1]
        # largest standard deviation; cap 4 sigma at n_map / 2
        tr, det = sxx + syy, sxx * syy - sxy * sxy
        lmax = 0.5 * tr + torch.sqrt(torch.clamp(0.25 * tr * tr - det, min=0.0))
        cap = (n_map / 8.0) ** 2
        scale = torch.clamp(cap / lmax, max=1.0)
        sxx, syy, sxy = sxx * scale, syy * scale, sxy * scale
        # light uniform on the hemisphere, view = towards the camera
        z = ud(a.numel(), 0.0, 1.0)
        ph = ud(a.numel(), 0.0, 2 * math.pi)
        r = torch.sqrt(1 - z * z)
        light = torch.stack([r * torch.cos(ph), r * torch.sin(ph), z], 1)
        view = -d / torch.linalg.vector_norm(d, dim=1, keepdim=True)
        h = light + view
        h = h / torch.linalg.vector_norm(h, dim=1, keepdim=True).clamp(min=1e-12)
        q = torch.stack([hit[:, 0] * n_map, hit[:, 1] * n_map, sxx, sxy, syy, h[:, 0], h[:, 1],
                         torch.zeros_like(sxx)], 1)
        out.append(q)
        need -= q.shape[0]
    return torch.cat(out)[:nq].to(torch.float32).contiguous()


def serving_maps(device="cpu"):
    """The four resident maps of the serving workload: 1024^2 bumps, 2048^2
    scratches, 4096^2 and 8192^2 flakes (fp32 (s, t))."""
    return [bumps_map(n=1024, n_bumps=1024, seed=11, device=device),
            scratch_map(n=2048, n_grooves=2000, seed=12, device=device),
            flake_map(n=4096, n_cells=50_000, seed=13, device=device),
            flake_map(n=8192, n_cells=200_000, seed=14, device=device)]


def serving_batches(n_batches: int, seed: int, sizes=(1000, 1_000_000)):
    """(map index, batch size, camera seed) per batch: size log-uniform in
    `sizes`, map uniform over the four serving maps."""
    g = _cpu_gen(seed, 70)
    n = torch.exp(_u(g, n_batches, math.log(sizes[0]), math.log(sizes[1]))).round().long()
    maps = torch.randint(0, 4, (n_batches,), generator=g)
    return [(int(maps[k]), int(n[k]), seed * 100_000 + k) for k in range(n_batches)]
