"""Seeded synthetic inputs shared by the oracle tests, the CUDA parity tests and
the benchmark.

This module holds geometry, radar-band and random-number set-up only (array
positions, cube and grid descriptors, network initial weights, scene
primitives, upstream gradients). It holds none of the rendering arithmetic, so
importing it couples neither the oracle to the CUDA path nor the reverse.

The workloads follow the paper's geometry (near field, 0.1-0.5 m, 77-81 GHz,
mm-pitch planar virtual arrays; App. C "Data Collection Setup") with synthetic
scenes standing in for the authors' unreleased radar captures.
"""
from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

# Primitive kinds of an analytic scene (values shared with the C-ABI header).
PRIM_SPHERE = 0      # p = (radius, -, -)
PRIM_BOX = 1         # p = half extents
PRIM_ELLIPSOID = 2   # p = radii
PRIM_HALFSPACE = 3   # c = point on the plane, p = unit normal towards free space

SAMPLE_UNIFORM = 0
SAMPLE_STRATIFIED = 1


@dataclass
class Grid:
    """Axis-aligned sample grid: n[0] x n[1] primary columns, n[2] depths.

    Point (ix, iy, k) has ray index iy*n[0] + ix and point index
    k*n_ray + ray (depth-major). ``aperture_z`` is the plane of the primary
    rays' start points (the array plane).
    """
    lo: Tuple[float, float, float]
    pitch: Tuple[float, float, float]
    n: Tuple[int, int, int]
    aperture_z: float = 0.0

    @property
    def n_ray(self) -> int:
        return self.n[0] * self.n[1]

    @property
    def n_pts(self) -> int:
        return self.n_ray * self.n[2]

    def lo32(self):
        return np.asarray(self.lo, dtype=np.float32)

    def pitch32(self):
        return np.asarray(self.pitch, dtype=np.float32)


def cube_grid(center, side, n, aperture_z=0.0) -> Grid:
    """Grid of n[0] x n[1] x n[2] cells over a cube of edge ``side``."""
    n = (int(n[0]), int(n[1]), int(n[2]))
    lo = tuple(float(np.float32(center[d] - side / 2.0)) for d in range(3))
    pitch = tuple(float(np.float32(side / n[d])) for d in range(3))
    return Grid(lo=lo, pitch=pitch, n=n, aperture_z=float(np.float32(aperture_z)))


def antenna_array(nx, ny, pitch, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Planar monostatic virtual array in the plane z = center[2], centred on
    center, FP32 SoA [3, nx*ny], antenna index iy*nx + ix."""
    ix = np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0
    iy = np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0
    X, Y = np.meshgrid(ix * pitch + center[0], iy * pitch + center[1], indexing="xy")
    out = np.empty((3, nx * ny), dtype=np.float32)
    out[0] = X.reshape(-1)
    out[1] = Y.reshape(-1)
    out[2] = center[2]
    return out


@dataclass
class Band:
    """Stepped frequencies f_n = f0 + n*df, n < n_f (FP64)."""
    f0: float
    df: float
    n_f: int


def fmcw_band(f_start=77e9, slope=70.15e12, fs=1.25e6, n_samples=64) -> Band:
    """FMCW chirp seen as stepped frequencies: ADC sample n at t_n = n / fs has
    the instantaneous frequency f_start + slope * t_n (section 3, Eq. fmcw).
    Defaults are the paper's radar (App. C): 77 GHz start, 70.15 MHz/us slope,
    64 samples at 1.25 Msps."""
    return Band(f0=float(f_start), df=float(slope / fs), n_f=int(n_samples))


def multi_plane_array(n_planes, nx, ny, pitch, radius, center=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Virtual arrays on n_planes scanning planes around an object (App. C: the
    object turns on a platform in front of a radar the arm sweeps over a 2-D
    aperture): plane m is an nx x ny array at `pitch`, its centre at distance
    `radius` from `center` in direction (sin t_m, 0, cos t_m), t_m = 2 pi m /
    n_planes, facing the centre (array axes: horizontal (cos t_m, 0, -sin t_m)
    and vertical (0, 1, 0)). FP32 SoA [3, n_planes*nx*ny], plane-major."""
    ix = np.arange(nx, dtype=np.float64) - (nx - 1) / 2.0
    iy = np.arange(ny, dtype=np.float64) - (ny - 1) / 2.0
    X, Y = np.meshgrid(ix * pitch, iy * pitch, indexing="xy")
    X, Y = X.reshape(-1), Y.reshape(-1)
    c = np.asarray(center, np.float64)
    out = []
    for m in range(n_planes):
        t = 2.0 * np.pi * m / n_planes
        nrm = np.array([np.sin(t), 0.0, np.cos(t)])
        hor = np.array([np.cos(t), 0.0, -np.sin(t)])
        ver = np.array([0.0, 1.0, 0.0])
        out.append(c[:, None] + radius * nrm[:, None] + hor[:, None] * X + ver[:, None] * Y)
    return np.concatenate(out, axis=1).astype(np.float32)


def band(f_lo=77e9, f_hi=81e9, n_f=32) -> Band:
    """n_f frequencies spanning [f_lo, f_hi], both end points included."""
    return Band(f0=float(f_lo), df=float((f_hi - f_lo) / (n_f - 1)), n_f=int(n_f))


@dataclass
class Prim:
    kind: int
    a: float
    c: Tuple[float, float, float]
    p: Tuple[float, float, float]


@dataclass
class Scene:
    prims: List[Prim] = field(default_factory=list)

    def packed(self) -> np.ndarray:
        """FP32 records of 8 values: kind, a, c[3], p[3]."""
        out = np.zeros((len(self.prims), 8), dtype=np.float32)
        for k, pr in enumerate(self.prims):
            out[k] = [pr.kind, pr.a, *pr.c, *pr.p]
        return out


@dataclass
class MLPSpec:
    """SDF + reflectiveness network: PE with ``n_levels`` octaves over a cube
    (x normalised by (x - center)/half), ``n_hidden`` softplus layers of
    ``width`` units, head [f, a_logit] (``head_out`` = 2), or a single output
    (``head_out`` = 1) for one of the two separate networks of FieldNets."""
    n_levels: int = 6
    width: int = 128
    n_hidden: int = 4
    beta: float = 100.0
    center: Tuple[float, float, float] = (0.0, 0.0, 0.15)
    half: float = 0.05
    head_out: int = 2

    @property
    def in_dim(self) -> int:
        return 6 * self.n_levels

    def shapes(self):
        dims = [self.in_dim] + [self.width] * self.n_hidden
        out = [(dims[l + 1], dims[l]) for l in range(self.n_hidden)]
        out.append((self.head_out, self.width))
        return out

    @property
    def n_params(self) -> int:
        return sum(o * i + o for o, i in self.shapes())


def mlp_init(spec: MLPSpec, seed: int, sdf_bias: float = 0.0) -> np.ndarray:
    """Packed FP32 parameters [W1 b1 W2 b2 ... W_head b_head], W row-major
    [out, in], U(-1/sqrt(fan_in), 1/sqrt(fan_in)) from a seeded generator.
    ``sdf_bias`` is added to the head's f bias."""
    rng = np.random.default_rng(seed)
    parts = []
    for li, (o, i) in enumerate(spec.shapes()):
        bound = 1.0 / np.sqrt(i)
        W = rng.uniform(-bound, bound, size=(o, i))
        b = rng.uniform(-bound, bound, size=(o,))
        if li == spec.n_hidden:
            b[0] += sdf_bias
        parts += [W.reshape(-1), b]
    return np.concatenate(parts).astype(np.float32)


@dataclass
class FieldNets:
    """The paper's two field networks (App. C): an SDF network (head [f]) and a
    separate reflectivity network (head [a_logit], a = sigmoid), both on the
    positional encoding of x; packed parameters [SDF network | reflectivity
    network], each packed like MLPSpec."""
    sdf: MLPSpec
    refl: MLPSpec

    @property
    def n_params(self) -> int:
        return self.sdf.n_params + self.refl.n_params


def paper_nets(center=(0.0, 0.0, 0.15), half=0.06, beta=100.0) -> FieldNets:
    """SDF network 8 x 256, reflectivity network 4 x 256, 10-octave encoding
    (App. C, "Training Setup"; softplus(beta) in both, a reading)."""
    return FieldNets(MLPSpec(10, 256, 8, beta, tuple(center), half, 1),
                     MLPSpec(10, 256, 4, beta, tuple(center), half, 1))


def nets_init(nets: FieldNets, seed: int, sdf_bias: float = 0.0) -> np.ndarray:
    return np.concatenate([mlp_init(nets.sdf, seed, sdf_bias), mlp_init(nets.refl, seed + 1000)])


def unpack_params(spec: MLPSpec, params: np.ndarray):
    """Views [(W, b), ...] into a packed parameter vector."""
    out, off = [], 0
    for o, i in spec.shapes():
        W = params[off:off + o * i].reshape(o, i); off += o * i
        b = params[off:off + o]; off += o
        out.append((W, b))
    assert off == params.size
    return out


def complex_normal(rng, shape, scale=1.0) -> np.ndarray:
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * (scale / np.sqrt(2.0))


# --- the five workloads ------------------------------------------------------

def c1_scene() -> Scene:
    """Sphere r = 3 cm at 15 cm range, reflectiveness 1."""
    return Scene([Prim(PRIM_SPHERE, 1.0, (0.0, 0.0, 0.15), (0.03, 0.0, 0.0))])


def c1_point_reflector(grid: Grid):
    """Isotropic point reflector at the centre of voxel (24, 16, 6) of the 32^3
    grid, outside the sphere; returned as FP32 xyz."""
    ijk = (24, 16, 6)
    return np.array([np.float32(np.float64(grid.lo[d]) + (ijk[d] + 0.5) * np.float64(grid.pitch[d]))
                     for d in range(3)], dtype=np.float32)


C4_OCCLUDER_Z = 0.10       # thin dielectric occluder plane between the array and the objects
C4_OCCLUDER_ATTEN = 0.5    # round-trip amplitude factor behind it
C4_SNR_DB = 10.0


def c4_noise(seed: int, shape, signal_power: float) -> np.ndarray:
    """Complex Gaussian noise of power signal_power / 10^(SNR/10), seeded."""
    rng = np.random.default_rng(10_000 + seed)
    return complex_normal(rng, shape, scale=np.sqrt(signal_power / 10.0 ** (C4_SNR_DB / 10.0)))


def c4_scene(seed: int, center=(0.0, 0.0, 0.15), side=0.12) -> Scene:
    """1-8 random ellipsoids and boxes, axes U[1, 4] cm, reflectiveness
    U[0.2, 1], centres inside the cube shrunk by the largest axis."""
    rng = np.random.default_rng(seed)
    prims = []
    for _ in range(int(rng.integers(1, 9))):
        kind = PRIM_ELLIPSOID if rng.uniform() < 0.5 else PRIM_BOX
        axes = rng.uniform(0.01, 0.04, 3)          # full axes; radii / half extents are half of them
        ext = axes / 2.0
        lim = side / 2.0 - ext.max()
        c = tuple(float(center[d] + rng.uniform(-lim, lim)) for d in range(3))
        prims.append(Prim(kind, float(rng.uniform(0.2, 1.0)), c, tuple(float(v) for v in ext)))
    return Scene(prims)


@dataclass
class Workload:
    name: str
    array_n: int
    array_pitch: float
    n_f: int
    grid: Grid
    heat: Grid
    sample_mode: int
    field: str            # "analytic" or "mlp"
    precision: str        # "fp32" or "bf16"
    sharpness: float
    a_tx: float = 1.0


def workload(name: str) -> Workload:
    """Sizes of the five workloads (sphere+point analytic 32^3; MLP 128^3; BF16
    MLP 256^3; training step 2^24; proposal 2^20)."""
    if name == "c1":
        g = cube_grid((0.0, 0.0, 0.15), 0.10, (32, 32, 32))
        return Workload(name, 16, 0.002, 32, g, g, SAMPLE_UNIFORM, "analytic", "fp32",
                        sharpness=2.0 / g.pitch[2])
    if name == "c2":
        g = cube_grid((0.0, 0.0, 0.15), 0.10, (128, 128, 128))
        h = cube_grid((0.0, 0.0, 0.15), 0.10, (64, 64, 64))
        return Workload(name, 64, 0.002, 128, g, h, SAMPLE_STRATIFIED, "mlp", "fp32",
                        sharpness=2.0 / h.pitch[2])
    if name == "c2-small":
        # same array, band and network as c2 with 1/32 of the samples (profiling size)
        g = cube_grid((0.0, 0.0, 0.15), 0.10, (64, 64, 16))
        h = cube_grid((0.0, 0.0, 0.15), 0.10, (32, 32, 32))
        return Workload(name, 64, 0.002, 128, g, h, SAMPLE_STRATIFIED, "mlp", "fp32",
                        sharpness=2.0 / h.pitch[2])
    if name == "c3":
        g = cube_grid((0.0, 0.0, 0.15), 0.10, (256, 256, 256))
        h = cube_grid((0.0, 0.0, 0.15), 0.10, (64, 64, 64))
        return Workload(name, 128, 0.002, 256, g, h, SAMPLE_STRATIFIED, "mlp", "bf16",
                        sharpness=2.0 / h.pitch[2])
    if name == "c3-small":
        # same array, band and network as c3 with 1/256 of the samples (profiling size)
        g = cube_grid((0.0, 0.0, 0.15), 0.10, (64, 64, 16))
        h = cube_grid((0.0, 0.0, 0.15), 0.10, (32, 32, 32))
        return Workload(name, 128, 0.002, 256, g, h, SAMPLE_STRATIFIED, "mlp", "bf16",
                        sharpness=2.0 / h.pitch[2])
    if name == "c4":
        g = cube_grid((0.0, 0.0, 0.15), 0.12, (256, 256, 256))
        h = cube_grid((0.0, 0.0, 0.15), 0.12, (64, 64, 64))
        return Workload(name, 64, 0.002, 128, g, h, SAMPLE_STRATIFIED, "mlp", "fp32",
                        sharpness=2.0 / h.pitch[2])
    if name == "c4-small":
        g = cube_grid((0.0, 0.0, 0.15), 0.12, (32, 32, 32))
        h = cube_grid((0.0, 0.0, 0.15), 0.12, (16, 16, 16))
        return Workload(name, 8, 0.004, 16, g, h, SAMPLE_STRATIFIED, "mlp", "fp32",
                        sharpness=2.0 / h.pitch[2])
    raise KeyError(name)
