"""Seeded synthetic inputs for the SEM Q-isosurface render path.

This module serves both the CPU oracle (``oracle/``) and the CUDA library
(``paper_2312_09888_gb300``): the tests and ``bench.py`` draw every input from here.
It holds none of the method's arithmetic -- no spectral derivative, no
Q-criterion, no marching cubes, no rasteriser.  It only

* places the sample points of a box mesh of hexahedral spectral elements
  (Gauss-Lobatto-Legendre points, taken from numpy's Legendre module),
* evaluates analytic velocity / scalar fields at those points, and
* describes the cameras and isovalue fractions of each workload.

The paper runs NekRS on its own pb146 and Rayleigh-Benard cases (Sec. 4.1,
4.2); those meshes and fields are not available, so the synthetic fields
below stand in for them with the element counts and polynomial order of each
workload.

Layouts (the library's and the oracle's common contract):

* elements are ordered ``e = ex + nex*(ey + ney*ez)``;
* the (N+1)^3 nodes of an element are ordered ``n = i + (N+1)*(j + (N+1)*k)``
  (r fastest), i.e. an element is ``u[e][k][j][i]``;
* node coordinates are SoA: ``xyz[0|1|2][e][n]``; fields are ``f[e][n]``.

Seeds: ``BASE_SEED + 1000*config_index + snapshot`` with numpy ``default_rng``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

BASE_SEED = 2312_09888


def seed_for(config_index: int, snapshot: int = 0) -> int:
    return BASE_SEED + 1000 * config_index + snapshot


def gll_points(N: int) -> np.ndarray:
    """Gauss-Lobatto-Legendre points on [-1, 1]: -1, the roots of P_N', +1.

    Uses numpy's Legendre class (a library routine), so that the sample points do
    not come from either implementation under test.
    """
    if N < 1:
        raise ValueError("N must be >= 1")
    if N == 1:
        return np.array([-1.0, 1.0])
    inner = np.polynomial.legendre.Legendre.basis(N).deriv().roots()
    inner = np.sort(np.real(inner))
    return np.concatenate([[-1.0], inner, [1.0]])


@dataclass
class BoxMesh:
    """Tensor-product mesh of affine hexahedra; element faces at xf, yf, zf."""

    N: int
    xf: np.ndarray
    yf: np.ndarray
    zf: np.ndarray

    @property
    def NP(self) -> int:
        return self.N + 1

    @property
    def nex(self) -> int:
        return len(self.xf) - 1

    @property
    def ney(self) -> int:
        return len(self.yf) - 1

    @property
    def nez(self) -> int:
        return len(self.zf) - 1

    @property
    def E(self) -> int:
        return self.nex * self.ney * self.nez

    def axis_points(self, faces: np.ndarray) -> np.ndarray:
        """Global 1-D node coordinates along one axis (shared face nodes once)."""
        xi = gll_points(self.N)
        pts = [faces[0]]
        for a, b in zip(faces[:-1], faces[1:]):
            loc = a + (xi + 1.0) * 0.5 * (b - a)
            loc[-1] = b
            pts.extend(loc[1:])
        return np.asarray(pts, dtype=np.float64)

    def global_axes(self):
        return self.axis_points(self.xf), self.axis_points(self.yf), self.axis_points(self.zf)

    def global_shape(self):
        return (self.nez * self.N + 1, self.ney * self.N + 1, self.nex * self.N + 1)

    def flat_index(self, device="cpu") -> torch.Tensor:
        """(E, NP^3) int64 index of each element node into the global grid
        laid out [iz][iy][ix]."""
        NP, N = self.NP, self.N
        e = torch.arange(self.E, device=device, dtype=torch.int64)
        ex = e % self.nex
        ey = (e // self.nex) % self.ney
        ez = e // (self.nex * self.ney)
        n = torch.arange(NP ** 3, device=device, dtype=torch.int64)
        i = n % NP
        j = (n // NP) % NP
        k = n // (NP * NP)
        nx = self.nex * N + 1
        ny = self.ney * N + 1
        ix = ex[:, None] * N + i[None, :]
        iy = ey[:, None] * N + j[None, :]
        iz = ez[:, None] * N + k[None, :]
        return ix + nx * (iy + ny * iz)

    def gather(self, g: torch.Tensor, idx: Optional[torch.Tensor] = None) -> torch.Tensor:
        """Global-grid field [iz][iy][ix] -> element layout (E, NP^3)."""
        if idx is None:
            idx = self.flat_index(g.device)
        return g.reshape(-1)[idx]

    def xyz(self, device="cpu") -> torch.Tensor:
        """(3, E, NP^3) float64 node coordinates."""
        gx, gy, gz = (torch.as_tensor(a, dtype=torch.float64, device=device) for a in self.global_axes())
        nz, ny, nx = self.global_shape()
        idx = self.flat_index(device)
        X = gx[None, None, :].expand(nz, ny, nx)
        Y = gy[None, :, None].expand(nz, ny, nx)
        Z = gz[:, None, None].expand(nz, ny, nx)
        return torch.stack([self.gather(X.contiguous(), idx), self.gather(Y.contiguous(), idx),
                            self.gather(Z.contiguous(), idx)])

    def xyz_range(self, e0: int, e1: int) -> np.ndarray:
        """(3, e1-e0, NP^3) float64 node coordinates of elements [e0, e1) only (the same values
        as xyz()[:, e0:e1], without building the whole mesh)."""
        gx, gy, gz = self.global_axes()
        NP, N = self.NP, self.N
        e = np.arange(e0, e1, dtype=np.int64)
        ex, ey, ez = e % self.nex, (e // self.nex) % self.ney, e // (self.nex * self.ney)
        n = np.arange(NP ** 3, dtype=np.int64)
        i, j, k = n % NP, (n // NP) % NP, n // (NP * NP)
        return np.stack([gx[ex[:, None] * N + i[None, :]], gy[ey[:, None] * N + j[None, :]],
                         gz[ez[:, None] * N + k[None, :]]])

    def grids(self, device="cpu"):
        """Broadcastable global coordinate grids X[1,1,nx], Y[1,ny,1], Z[nz,1,1]."""
        gx, gy, gz = (torch.as_tensor(a, dtype=torch.float64, device=device) for a in self.global_axes())
        return gx[None, None, :], gy[None, :, None], gz[:, None, None]


def perturbed_box(n: Sequence[int], lo: Sequence[float], hi: Sequence[float], N: int, amp: float = 0.2,
                  seed: int = 0) -> np.ndarray:
    """(3, E, NP^3) float64 node coordinates of a conforming curved mesh: the uniform grid of
    element corners with every interior corner moved by up to amp times the element size per
    axis (seeded; a grid with a single element along some axis has no interior corner and stays
    a box), each element the trilinear map of its eight corners sampled at the GLL points.  Element order e = ex + nx (ey + ny ez), node order i + NP (j + NP k), as in
    BoxMesh."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n
    h = [(hi[d] - lo[d]) / n[d] for d in range(3)]
    cx, cy, cz = (np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3))
    C = np.stack(np.meshgrid(cx, cy, cz, indexing="ij"), axis=-1)  # (nx+1, ny+1, nz+1, 3)
    inner = (slice(1, nx), slice(1, ny), slice(1, nz))
    C[inner] += rng.uniform(-amp, amp, size=C[inner].shape) * np.array(h)
    xi = gll_points(N)
    NP = N + 1
    r = np.broadcast_to(xi[None, None, :], (NP, NP, NP)).reshape(-1)
    s_ = np.broadcast_to(xi[None, :, None], (NP, NP, NP)).reshape(-1)
    t = np.broadcast_to(xi[:, None, None], (NP, NP, NP)).reshape(-1)
    xyz = np.zeros((3, nx * ny * nz, NP ** 3))
    for ez in range(nz):
        for ey in range(ny):
            for ex in range(nx):
                e = ex + nx * (ey + ny * ez)
                for v in range(8):
                    a, b, c = v & 1, (v >> 1) & 1, (v >> 2) & 1
                    wgt = ((1 + r) / 2 if a else (1 - r) / 2) * ((1 + s_) / 2 if b else (1 - s_) / 2) * \
                          ((1 + t) / 2 if c else (1 - t) / 2)
                    xyz[:, e] += C[ex + a, ey + b, ez + c][:, None] * wgt[None, :]
    return xyz


def uniform_box(n: Sequence[int], lo: Sequence[float], hi: Sequence[float], N: int) -> BoxMesh:
    f = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
    return BoxMesh(N, f[0], f[1], f[2])


# --------------------------------------------------------------------------- fields

def taylor_green(mesh: BoxMesh, noise_sigma: float = 0.0, seed: int = 0, device="cpu",
                 phase: float = 0.0) -> torch.Tensor:
    """(3, E, NP^3) float64: u = sin x cos y cos z, v = -cos x sin y cos z, w = 0,
    shifted by ``phase`` in x and y, plus i.i.d. N(0, sigma^2) per global node
    (shared face nodes get the same sample, so the field stays continuous)."""
    X, Y, Z = mesh.grids(device)
    shape = mesh.global_shape()
    Xp, Yp = X + phase, Y + phase
    u = (torch.sin(Xp) * torch.cos(Yp) * torch.cos(Z)).expand(shape)
    v = (-torch.cos(Xp) * torch.sin(Yp) * torch.cos(Z)).expand(shape)
    w = torch.zeros(shape, dtype=torch.float64, device=device)
    comps = [u.contiguous(), v.contiguous(), w]
    if noise_sigma > 0.0:
        rng = np.random.default_rng(seed)
        noise = rng.normal(0.0, noise_sigma, size=(3,) + shape)
        nt = torch.as_tensor(noise, device=device)
        comps = [c + nt[d] for d, c in enumerate(comps)]
    idx = mesh.flat_index(device)
    return torch.stack([mesh.gather(c, idx) for c in comps])


def taylor_green_snapshots(mesh: BoxMesh, E: int, phases, noise_sigma: float, seed: int,
                           device="cuda") -> list:
    """The snapshots of the batching workload: for each phase, (3, E, NP^3) float32 of the first
    E elements of ``mesh`` holding taylor_green()'s field (u = sin x cos y cos z, v = -cos x sin y
    cos z, w = 0, shifted by the phase in x and y) plus i.i.d. N(0, sigma^2) noise per global node
    (shared face nodes share the sample).  The noise comes from torch's generator seeded with
    ``seed`` on the device rather than numpy's on the host, so 64 snapshots of 16 partitions take
    seconds; the values therefore differ from taylor_green()'s for the same seed, not their law."""
    X, Y, Z = mesh.grids(device)
    shape = mesh.global_shape()
    idx = mesh.flat_index(device)[:E]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    out = []
    for ph in phases:
        Xp, Yp = X + ph, Y + ph
        base = [torch.sin(Xp) * torch.cos(Yp) * torch.cos(Z), -torch.cos(Xp) * torch.sin(Yp) * torch.cos(Z), None]
        comps = []
        for c in range(3):
            f = torch.randn(shape, generator=g, device=device, dtype=torch.float64) * noise_sigma
            if base[c] is not None:
                f += base[c]
            comps.append(f.reshape(-1)[idx].float())
        out.append(torch.stack(comps))
    return out


def _random_modes(rng, nmodes, kmin, kmax, int_x, int_y, even_z):
    ks, amps, dirs, phases = [], [], [], []
    for _ in range(nmodes):
        kmag = rng.uniform(kmin, kmax)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        k = kmag * d
        if int_x:
            k[0] = np.round(k[0])
        if int_y:
            k[1] = np.round(k[1])
        if even_z:
            k[2] = 2.0 * np.round(k[2] / 2.0)
        if np.linalg.norm(k) == 0.0:
            k[1] = 1.0
        a = rng.normal(size=3)
        a -= k * (a @ k) / (k @ k)
        a /= np.linalg.norm(a)
        ks.append(k)
        amps.append(np.linalg.norm(k) ** (-5.0 / 6.0))
        dirs.append(a)
        phases.append(rng.uniform(0.0, 2.0 * np.pi))
    return np.array(ks), np.array(amps), np.array(dirs), np.array(phases)


def _sum_modes(mesh: BoxMesh, ks, amps, dirs, phases, device, phase_shift=0.0):
    """sum_m amps_m dirs_m cos(k_m . x + phases_m) on the global grid, per component.

    Each mode is separable, cos(a+b+c) = Re(e^{ia} e^{ib} e^{ic}), so the sum is a
    rank-M product evaluated slab by slab."""
    gx, gy, gz = (torch.as_tensor(a, dtype=torch.float64, device=device) for a in mesh.global_axes())
    k = torch.as_tensor(ks, device=device)
    ph = torch.as_tensor(phases, device=device) + phase_shift
    Ex = torch.exp(1j * (gx[:, None] * k[None, :, 0] + ph[None, :])) * torch.as_tensor(amps, device=device)[None, :]
    Ey = torch.exp(1j * (gy[:, None] * k[None, :, 1]))
    Ez = torch.exp(1j * (gz[:, None] * k[None, :, 2]))
    d = torch.as_tensor(dirs, device=device).to(torch.complex128)
    nz, ny, nx = len(gz), len(gy), len(gx)
    out = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=device)
    ExT = Ex.T.contiguous()
    zc = max(1, (1 << 22) // max(1, ny * len(phases)))
    for z0 in range(0, nz, zc):
        z1 = min(nz, z0 + zc)
        A = Ez[z0:z1, None, :] * Ey[None, :, :]          # (zc, ny, M)
        for c in range(3):
            T = (A * d[None, None, :, c]).reshape(-1, len(phases)) @ ExT
            out[c, z0:z1] = T.real.reshape(z1 - z0, ny, nx)
    return out


def channel_flow(mesh: BoxMesh, nmodes: int = 512, seed: int = 0, device="cpu",
                 rms: float = 0.1) -> torch.Tensor:
    """(3, E, NP^3) float64 channel field on [0,2pi] x [-1,1] x [0,pi]:
    u = (1-y^2) e_x + (1-y^2) * s * sum_m A_m a_m cos(k_m.x + phi_m), with
    |k| ~ U[1,32], k_x integer, k_z even (periodic), a_m perpendicular to k_m,
    A_m = |k_m|^(-5/6) (a k^-5/3 energy spectrum) and s chosen so that the
    fluctuation has rms ``rms`` over the grid."""
    rng = np.random.default_rng(seed)
    ks, amps, dirs, phases = _random_modes(rng, nmodes, 1.0, 32.0, True, False, True)
    F = _sum_modes(mesh, ks, amps, dirs, phases, device)
    F *= rms / torch.sqrt(torch.mean(F * F))
    X, Y, Z = mesh.grids(device)
    damp = (1.0 - Y * Y)
    comps = [damp * (1.0 + F[0]), damp * F[1], damp * F[2]]
    idx = mesh.flat_index(device)
    return torch.stack([mesh.gather(c.expand(mesh.global_shape()).contiguous(), idx) for c in comps])


def rayleigh_benard(mesh: BoxMesh, nmodes: int = 64, seed: int = 0, device="cpu",
                    amp: float = 0.1):
    """(4, E, NP^3) float64 on [0,2pi]^2 x [0,1]: convection rolls with k=3,
    u = (pi/3) sin3x cos(pi z), v = (pi/3) sin3y cos(pi z),
    w = -(cos3x + cos3y) sin(pi z) (divergence free), temperature
    T = 1 - z + 0.1 (cos3x + cos3y) sin(pi z), each plus ``nmodes`` seeded random
    modes of rms ``amp``.  Returns u, v, w, T."""
    rng = np.random.default_rng(seed)
    ks, amps, dirs, phases = _random_modes(rng, nmodes, 1.0, 16.0, True, True, False)
    F = _sum_modes(mesh, ks, amps, dirs, phases, device)
    F *= amp / torch.sqrt(torch.mean(F * F))
    X, Y, Z = mesh.grids(device)
    shape = mesh.global_shape()
    pz = math.pi * Z
    u = (math.pi / 3) * torch.sin(3 * X) * torch.cos(pz) + F[0]
    v = (math.pi / 3) * torch.sin(3 * Y) * torch.cos(pz) + F[1]
    w = -(torch.cos(3 * X) + torch.cos(3 * Y)) * torch.sin(pz) + F[2]
    T = 1.0 - Z + 0.1 * (torch.cos(3 * X) + torch.cos(3 * Y)) * torch.sin(pz) + (F[0] + F[1] + F[2]) / 3.0
    idx = mesh.flat_index(device)
    return torch.stack([mesh.gather(c.expand(shape).contiguous(), idx) for c in (u, v, w, T)])


def sphere_field(mesh: BoxMesh, center, radius: float, device="cpu") -> torch.Tensor:
    """(E, NP^3) float64: |x - c|^2 - r^2 (a degree-2 polynomial per direction)."""
    X, Y, Z = mesh.grids(device)
    g = (X - center[0]) ** 2 + (Y - center[1]) ** 2 + (Z - center[2]) ** 2 - radius ** 2
    return mesh.gather(g.expand(mesh.global_shape()).contiguous())


# --------------------------------------------------------------------------- cameras

def camera(ortho: bool, eye, center, up, W: int, H: int, fovy_deg: float = 40.0,
           half_h: float = 1.0, znear: float = 0.1, zfar: float = 100.0) -> dict:
    return dict(ortho=int(ortho), eye=[float(v) for v in eye], center=[float(v) for v in center],
                up=[float(v) for v in up], fovy_deg=float(fovy_deg), half_h=float(half_h),
                znear=float(znear), zfar=float(zfar), W=int(W), H=int(H))


def box_camera_ortho(lo, hi, W, H, direction=(1.0, 1.0, 1.0), up=(0.0, 0.0, 1.0)) -> dict:
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    c = (lo + hi) / 2
    R = float(np.linalg.norm(hi - lo) / 2)
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    eye = c + 2.0 * R * d
    return camera(True, eye, c, up, W, H, half_h=R, znear=R * 0.5, zfar=R * 4.0)


def box_camera_persp(lo, hi, W, H, direction=(1.0, 0.8, 1.2), up=(0.0, 1.0, 0.0),
                     fovy_deg=40.0, dist=2.5) -> dict:
    lo, hi = np.asarray(lo, float), np.asarray(hi, float)
    c = (lo + hi) / 2
    R = float(np.linalg.norm(hi - lo) / 2)
    d = np.asarray(direction, float)
    d /= np.linalg.norm(d)
    eye = c + dist * R * d
    return camera(False, eye, c, up, W, H, fovy_deg=fovy_deg, znear=0.5 * R, zfar=(dist + 1.5) * R)


# --------------------------------------------------------------------------- workloads

TWO_PI = 2.0 * math.pi


@dataclass
class Workload:
    name: str
    index: int
    mesh: BoxMesh
    iso_fracs: list
    camera: dict
    fields: Optional[torch.Tensor] = None       # (3 or 4, E, NP^3) float64
    extra: dict = field(default_factory=dict)

    @property
    def E(self):
        return self.mesh.E


def tgv_box(nel: int = 8, N: int = 7, W: int = 256, H: int = 256, noise: float = 1e-3,
            device="cpu", snapshot: int = 0, phase: float = 0.0) -> Workload:
    """Taylor-Green vortex on [0,2pi]^3 with nel^3 elements of order N, seeded
    1e-3 Gaussian noise, one Q-isosurface at 0.1*maxQ, orthographic camera
    looking from (1,1,1) at the centre, 256x256."""
    mesh = uniform_box((nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3, N)
    f = taylor_green(mesh, noise, seed_for(1, snapshot), device, phase=phase)
    cam = box_camera_ortho((0.0,) * 3, (TWO_PI,) * 3, W, H)
    return Workload(f"tgv_{nel}^3_N{N}", 1, mesh, [0.1], cam, f)


def channel_mesh(nel=(32, 32, 32), N: int = 7, stretch: float = 2.0) -> BoxMesh:
    eta = np.linspace(-1.0, 1.0, nel[1] + 1)
    yf = np.tanh(stretch * eta) / np.tanh(stretch)
    yf[0], yf[-1] = -1.0, 1.0
    return BoxMesh(N, np.linspace(0.0, TWO_PI, nel[0] + 1), yf, np.linspace(0.0, math.pi, nel[2] + 1))


def channel(nel=(32, 32, 32), N: int = 7, W: int = 1920, H: int = 1080, nmodes: int = 512,
            device="cpu", snapshot: int = 0) -> Workload:
    """Channel [0,2pi] x [-1,1] x [0,pi], wall-clustered element faces
    (tanh stretch 2.0), 512 seeded random Fourier modes with a k^-5/3
    spectrum damped by (1-y^2) plus a parabolic mean; Q-isosurfaces at
    {0.05, 0.1, 0.2}*maxQ; 1920x1080 perspective."""
    mesh = channel_mesh(nel, N)
    f = channel_flow(mesh, nmodes, seed_for(2, snapshot), device)
    cam = box_camera_persp((0.0, -1.0, 0.0), (TWO_PI, 1.0, math.pi), W, H)
    return Workload(f"channel_{nel[0]}x{nel[1]}x{nel[2]}_N{N}", 2, mesh, [0.05, 0.1, 0.2], cam, f)


def rb_box(nel: int = 64, N: int = 7, W: int = 3840, H: int = 2160, device="cpu",
           snapshot: int = 0) -> Workload:
    mesh = BoxMesh(N, np.linspace(0, TWO_PI, nel + 1), np.linspace(0, TWO_PI, nel + 1),
                   np.linspace(0, 1.0, nel + 1))
    f = rayleigh_benard(mesh, 64, seed_for(3, snapshot), device)
    cam = box_camera_persp((0.0, 0.0, 0.0), (TWO_PI, TWO_PI, 1.0), W, H,
                           direction=(1.0, -1.2, 0.8), up=(0.0, 0.0, 1.0))
    return Workload(f"rb_{nel}^3_N{N}", 3, mesh, [0.1], cam, f, extra=dict(t_iso=0.5))


def batching_partitions() -> list:
    """The batching workload's 16 partitions: E_p ~ U{4096..40960} elements and N_p in {5, 7, 9}
    (seeded), each the lexicographically first E_p elements of a ceil(E_p^(1/3))^3 lattice of
    [0, 2 pi]^3.  Returns dicts with E, N and mesh (the whole lattice; its first E elements are
    the partition)."""
    rng = np.random.default_rng(seed_for(4, 0))
    parts = []
    for _ in range(16):
        Ep, N = int(rng.integers(4096, 40961)), int(rng.choice([5, 7, 9]))
        n = int(math.ceil(Ep ** (1.0 / 3.0) - 1e-9))
        parts.append(dict(E=Ep, N=N, mesh=uniform_box((n, n, n), (0.0,) * 3, (TWO_PI,) * 3, N)))
    return parts


def element_slice(w: Workload, e0: int, e1: int) -> dict:
    """Contiguous element range [e0, e1) of a workload: node coordinates and fields."""
    xyz = w.mesh.xyz(w.fields.device)[:, e0:e1]
    return dict(xyz=xyz, fields=w.fields[:, e0:e1], N=w.mesh.N)


def random_nodal(mesh: BoxMesh, ncomp: int = 1, seed: int = 0, scale: float = 1.0) -> torch.Tensor:
    """(ncomp, E, NP^3) float64 i.i.d. N(0, scale^2) per element node (not continuous across
    elements; the derivative path is element-local)."""
    rng = np.random.default_rng(seed)
    return torch.as_tensor(rng.normal(0.0, scale, size=(ncomp, mesh.E, mesh.NP ** 3)))


def stretched_box(nel, N: int, seed: int = 0) -> BoxMesh:
    """Box mesh with seeded uneven element widths along each axis."""
    rng = np.random.default_rng(seed)
    faces = []
    for d, n in enumerate(nel):
        w = rng.uniform(0.5, 1.5, size=n)
        f = np.concatenate([[0.0], np.cumsum(w)]) - 0.3 * d
        faces.append(f)
    return BoxMesh(N, faces[0], faces[1], faces[2])


# --------------------------------------------------------------------------- learned compression

AE_DIMS = (1536, 512, 48, 512, 1536)   # per-element autoencoder widths (N = 7, 3 components)
AE_SNAPSHOTS_TRAIN = 200
AE_SNAPSHOTS_TOTAL = 250


def ae_init_params(seed: int = None, dims=AE_DIMS) -> dict:
    """Initial weights of the four layers: W_l ~ U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a
    seeded numpy generator, biases zero; float32 arrays W_l (out, in), b_l (out,)."""
    rng = np.random.default_rng(seed_for(5) if seed is None else seed)
    p = {}
    for layer in range(4):
        fin, fout = dims[layer], dims[layer + 1]
        a = 1.0 / math.sqrt(fin)
        p[f"W{layer + 1}"] = rng.uniform(-a, a, size=(fout, fin)).astype(np.float32)
        p[f"b{layer + 1}"] = np.zeros(fout, dtype=np.float32)
    return p


def ae_snapshot(s: int, nel: int = 32, N: int = 7, noise: float = 1e-3, device="cpu") -> torch.Tensor:
    """Snapshot s of the learned-compression data: the Taylor-Green field of the small
    workload on nel^3 elements, phase 2 pi s / 250 in x and y, plus i.i.d. N(0, noise^2) per
    global node (shared face nodes share the sample, as in the small workload), drawn from
    torch's generator on `device` seeded with seed_for(5, s).  Returns (3, E, (N+1)^3)
    float32 on `device` (noise-free when noise == 0)."""
    mesh = uniform_box((nel,) * 3, (0.0,) * 3, (TWO_PI,) * 3, N)
    f = taylor_green(mesh, 0.0, 0, device, phase=TWO_PI * s / AE_SNAPSHOTS_TOTAL)
    if noise > 0.0:
        g = torch.Generator(device=device)
        g.manual_seed(seed_for(5, s))
        nz = noise * torch.randn((3,) + mesh.global_shape(), generator=g, device=device, dtype=torch.float64)
        idx = mesh.flat_index(device)
        f = f + torch.stack([mesh.gather(nz[c], idx) for c in range(3)])
    return f.float()


def ae_samples(fields: torch.Tensor) -> torch.Tensor:
    """(3, E, NP^3) fields -> (E, 3 NP^3) samples [u_e | v_e | w_e] (a pure relayout)."""
    return fields.permute(1, 0, 2).reshape(fields.shape[1], -1).contiguous()
