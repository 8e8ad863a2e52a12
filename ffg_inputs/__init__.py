"""Seeded synthetic tuning spaces and runtimes.

This module only *describes* inputs: the parameter value lists of a tuning
space, the constraint clauses that a configuration must satisfy, and a
runtime (fitness) for every point of the full Cartesian product.  It holds
none of the method's arithmetic: it never decides which configuration is
valid, never enumerates neighbours, never builds a graph and never ranks
nodes.  Both the CPU oracle and the CUDA library consume what it produces.

Spaces follow the paper's definition (Sec. III-B): a space is the Cartesian
product X = S_1 x ... x S_n of finite integer value lists.  Runtimes are laid
out row-major over that product (parameter 0 is the slowest axis, the last
parameter the fastest), i.e. exactly ``numpy.ravel`` order of an array of
shape ``(len(S_1), ..., len(S_n))``.

The paper's own spaces come from brute-force cache files of real GPU runs
(Sec. V); they are not available, so the runtimes here are a seeded model
with the features those landscapes have: a smooth multimodal trend in the
log of the parameter values, measurement noise, and a fraction of points
that "failed" and carry the sentinel runtime 1e10 (Sec. V gives that value).

Random numbers are drawn from a counter-based generator (SplitMix64's
finaliser applied to ``base(seed, stream) + i * golden_gamma``), so each
value depends only on (seed, stream, index), never on evaluation order or
on the numpy version.

Clause kinds (the semantics that both consumers implement independently):

* ``prod_le``      prod(values[a]) <= bound
* ``prod_ge``      prod(values[a]) >= bound
* ``divides``      prod(values[a]) mod prod(values[b]) == 0   (false if the
                   divisor is 0)
* ``prod_le_prod`` prod(values[a]) <= prod(values[b])

An empty index tuple has product 1.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field

import numpy as np

FAIL_RUNTIME = 1e10          # sentinel runtime of a failed configuration (Sec. V)
CLAUSE_KINDS = ("prod_le", "prod_ge", "divides", "prod_le_prod")

_M64 = (1 << 64) - 1
_GAMMA = 0x9E3779B97F4A7C15


@dataclass(frozen=True)
class Clause:
    kind: str
    a: tuple = ()
    b: tuple = ()
    bound: int = 0

    def __post_init__(self):
        if self.kind not in CLAUSE_KINDS:
            raise ValueError(f"unknown clause kind {self.kind!r}")


@dataclass(frozen=True)
class SpaceSpec:
    """A tuning space: named integer value lists plus constraint clauses."""
    name: str
    names: tuple
    values: tuple
    clauses: tuple = field(default=())

    @property
    def n_params(self) -> int:
        return len(self.values)

    @property
    def radix(self) -> tuple:
        return tuple(len(v) for v in self.values)

    @property
    def n_raw(self) -> int:
        return int(np.prod(self.radix, dtype=np.int64)) if self.values else 0


# --------------------------------------------------------------------------
# counter-based random numbers
# --------------------------------------------------------------------------

def _mix64_int(z: int) -> int:
    z &= _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z ^ (z >> np.uint64(30))
    z = z * np.uint64(0xBF58476D1CE4E5B9)
    z = z ^ (z >> np.uint64(27))
    z = z * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> int:
    return _mix64_int((seed * 0x100000001B3) ^ ((stream + 1) * 0xC2B2AE3D27D4EB4F))


def uniform01(seed: int, stream: int, index) -> np.ndarray:
    """U[0,1) doubles keyed by (seed, stream, index); index is an int array."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(_base(seed, stream)) + (idx + np.uint64(1)) * np.uint64(_GAMMA)
        h = _mix64(z)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _uniform_n(seed: int, stream: int, n: int, lo: float, hi: float) -> np.ndarray:
    return lo + (hi - lo) * uniform01(seed, stream, np.arange(n))


# --------------------------------------------------------------------------
# runtime model
# --------------------------------------------------------------------------

def _coordinate(vals) -> np.ndarray:
    """z in [-1, 1] per list entry: log2 of positive numeric lists, else position."""
    v = np.asarray(vals, dtype=np.float64)
    u = np.log2(v) if np.all(v > 0) else np.arange(len(v), dtype=np.float64)
    span = u.max() - u.min()
    if span == 0:
        return np.zeros_like(u)
    return 2.0 * (u - u.min()) / span - 1.0


def runtimes(spec: SpaceSpec, seed: int, fail_frac: float = 0.03, noise_sd: float = 0.05,
             quantum: float | None = None, n_bumps: int = 3) -> np.ndarray:
    """Runtime of every point of the Cartesian product, float64, row-major.

    runtime = exp(1 + g(z) + eps) where
      g = sum_i a_i (z_i-m_i)^2 + sum_{i<j} b_ij (z_i-m_i)(z_j-m_j)
          - sum_k h_k exp(-|z-mu_k|^2 / (2 sigma_k^2)),
      a_i ~ U(0.2,1), m_i ~ U(-0.6,0.6), b_ij ~ U(-0.15,0.15),
      h_k ~ U(0.3,0.8), sigma_k ~ U(0.15,0.35), mu_k ~ U(-1,1)^n,
      eps ~ N(0, noise_sd^2) (Box-Muller on two counter streams).
    A fraction ``fail_frac`` of points (a Bernoulli draw per point) gets the
    failure runtime 1e10.  ``quantum`` rounds runtimes to that step, which
    creates plateaus of equal fitness (ties).
    """
    n = spec.n_params
    shape = spec.radix
    R = spec.n_raw
    z = [_coordinate(v) for v in spec.values]
    a = _uniform_n(seed, 1, n, 0.2, 1.0)
    m = _uniform_n(seed, 2, n, -0.6, 0.6)
    bij = _uniform_n(seed, 3, n * n, -0.15, 0.15).reshape(n, n)
    h = _uniform_n(seed, 4, n_bumps, 0.3, 0.8)
    sig = _uniform_n(seed, 5, n_bumps, 0.15, 0.35)
    mu = _uniform_n(seed, 6, n_bumps * n, -1.0, 1.0).reshape(n_bumps, n)

    def axis(i, vec):
        s = [1] * n
        s[i] = len(vec)
        return np.asarray(vec, dtype=np.float64).reshape(s)

    g = np.zeros(shape, dtype=np.float64)
    for i in range(n):
        g += axis(i, a[i] * (z[i] - m[i]) ** 2)
    for i in range(n):
        for j in range(i + 1, n):
            g += bij[i, j] * axis(i, z[i] - m[i]) * axis(j, z[j] - m[j])
    for k in range(n_bumps):
        bump = np.ones(shape, dtype=np.float64)
        for i in range(n):
            bump = bump * axis(i, np.exp(-((z[i] - mu[k, i]) ** 2) / (2.0 * sig[k] ** 2)))
        g -= h[k] * bump
    g = g.reshape(-1)

    idx = np.arange(R, dtype=np.uint64)
    u1 = uniform01(seed, 101, idx)
    u2 = uniform01(seed, 102, idx)
    eps = noise_sd * np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)
    rt = np.exp(1.0 + g + eps)
    if quantum is not None:
        rt = np.round(rt / quantum) * quantum
    if fail_frac > 0:
        fail = uniform01(seed, 103, idx) < fail_frac
        rt[fail] = FAIL_RUNTIME
    return rt


# --------------------------------------------------------------------------
# spaces shaped like the paper's and the measured configurations
# --------------------------------------------------------------------------

def _pow2(lo_exp: int, hi_exp: int) -> tuple:
    return tuple(1 << e for e in range(lo_exp, hi_exp + 1))


def single_small() -> SpaceSpec:
    """5-parameter 2-D block/tile space, 1,344 raw points, 32 <= bx*by <= 1024."""
    return SpaceSpec(
        "single_small_1344",
        ("block_size_x", "block_size_y", "tile_size_x", "tile_size_y", "use_smem"),
        (_pow2(4, 10), _pow2(0, 5), _pow2(0, 3), _pow2(0, 3), (0, 1)),
        (Clause("prod_le", (0, 1), (), 1024), Clause("prod_ge", (0, 1), (), 32)),
    )


def single_large() -> SpaceSpec:
    """9-parameter space, 2,162,688 raw points under three clauses."""
    return SpaceSpec(
        "single_large_2162688",
        ("block_size_x", "block_size_y", "tile_size_x", "tile_size_y", "vector",
         "unroll", "stages", "use_padding", "read_only"),
        ((16, 32, 48, 64, 80, 96, 112, 128, 256, 512, 1024), _pow2(0, 7),
         tuple(range(1, 9)), tuple(range(1, 9)), _pow2(0, 5), _pow2(0, 3), (1, 2, 3, 4),
         (0, 1), (0, 1)),
        (Clause("prod_le", (0, 1), (), 4096), Clause("prod_le", (0, 1, 2, 3), (), 65536),
         Clause("divides", (0, 2), (4,))),
    )


def precision_large() -> SpaceSpec:
    """single_large plus two unconstrained 3-valued parameters (11 params, 19.5M raw)."""
    base = single_large()
    return SpaceSpec(
        "precision_large_19464192",
        base.names + ("loop_order", "prefetch"),
        base.values + ((1, 2, 3), (0, 1, 2)),
        base.clauses,
    )


# The paper's three kernel spaces (appendix table of tunable parameters).
# The constraint clauses are this project's: the paper only reports that many
# points fail to compile, which the runtime model covers with ``fail_frac``.

def conv_space() -> SpaceSpec:
    return SpaceSpec(
        "convolution",
        ("block_size_x", "block_size_y", "tile_size_x", "tile_size_y", "use_padding", "read_only"),
        ((1, 2, 4, 8, 16, 32, 48, 64, 80, 96, 112, 128), _pow2(0, 5), tuple(range(1, 9)),
         tuple(range(1, 9)), (0, 1), (0, 1)),
        (Clause("prod_le", (0, 1), (), 1024), Clause("prod_ge", (0, 1), (), 32)),
    )


def conv_mi50_space() -> SpaceSpec:
    return SpaceSpec(
        "convolution_mi50",
        ("block_size_x", "block_size_y", "tile_size_x", "tile_size_y", "use_padding"),
        ((16, 32, 48, 64, 80, 96, 112, 128), _pow2(0, 5), (1, 2, 4), (1, 2, 4), (0, 1)),
        (),
    )


def gemm_space() -> SpaceSpec:
    return SpaceSpec(
        "gemm",
        ("MWG", "NWG", "MDIMC", "NDIMC", "MDIMA", "NDIMB", "VWM", "VWN", "SA", "SB"),
        (_pow2(4, 7), _pow2(4, 7), (8, 16, 32), (8, 16, 32), (8, 16, 32), (8, 16, 32),
         _pow2(0, 3), _pow2(0, 3), (0, 1), (0, 1)),
        (Clause("divides", (0,), (2, 6)), Clause("divides", (1,), (3, 7)),
         Clause("prod_le", (2, 3), (), 1024)),
    )


def pnpoly_space() -> SpaceSpec:
    return SpaceSpec(
        "pnpoly",
        ("block_size_x", "tile_size", "between_method", "use_precomputed_slopes", "use_method"),
        (tuple(range(32, 1024, 32)), (1,) + tuple(range(2, 21, 2)), (0, 1, 2, 3), (0, 1),
         (0, 1, 2)),
        (),
    )


PAPER_SPACES = {
    "convolution": (conv_space, 18432),
    "convolution_mi50": (conv_mi50_space, 864),
    "gemm": (gemm_space, 82944),
    "pnpoly": (pnpoly_space, 8184),
}


def random_space(seed: int, n_params: int, max_radix: int = 12, n_clauses: int = 2,
                 name: str | None = None) -> SpaceSpec:
    """A seeded random space: value lists of powers of two or small ranges,
    with ``n_clauses`` product/divisibility clauses whose bounds are drawn
    from the range of the clause's product."""
    u = lambda stream, n: uniform01(seed, stream, np.arange(n))  # noqa: E731
    r = 2 + np.floor(u(1, n_params) * (max_radix - 1)).astype(int)
    style = u(2, n_params)
    vals = []
    for i in range(n_params):
        k = int(r[i])
        if style[i] < 0.5:
            vals.append(tuple(1 << e for e in range(k)))
        elif style[i] < 0.8:
            vals.append(tuple(range(1, k + 1)))
        else:
            vals.append(tuple(range(k)))
    clauses = []
    cu = u(3, 8 * max(n_clauses, 1))
    for c in range(n_clauses):
        i = int(cu[8 * c] * n_params)
        j = int(cu[8 * c + 1] * n_params)
        if i == j:
            j = (i + 1) % n_params
        kind_u = cu[8 * c + 2]
        if i == j:  # one parameter: a single-factor bound
            bound = int(vals[i][int(cu[8 * c + 3] * len(vals[i]))])
            clauses.append(Clause("prod_le" if kind_u < 0.6 else "prod_ge", (i,), (), bound))
            continue
        lo = max(min(vals[i]), 1) * max(min(vals[j]), 1)
        hi = max(max(vals[i]), 1) * max(max(vals[j]), 1)
        frac = 0.35 + 0.5 * cu[8 * c + 3]
        bound = int(round(math.exp(math.log(lo) + frac * (math.log(hi) - math.log(lo))))) if hi > lo else hi
        if kind_u < 0.45:
            clauses.append(Clause("prod_le", (i, j), (), bound))
        elif kind_u < 0.7:
            clauses.append(Clause("prod_ge", (i, j), (), max(lo, bound // 4)))
        elif kind_u < 0.85 and all(v > 0 for v in vals[j]):
            clauses.append(Clause("divides", (i,), (j,)))
        else:
            clauses.append(Clause("prod_le_prod", (i,), (j,)))
    return SpaceSpec(name or f"random_{seed}", tuple(f"p{i}" for i in range(n_params)),
                     tuple(vals), tuple(clauses))


def sized_random_space(seed: int, target_raw: int, max_radix: int = 12) -> SpaceSpec:
    """Random space whose raw size lies close to ``target_raw``: radices are
    drawn one parameter at a time until the product reaches the target.
    Clauses: a product upper bound on one pair of parameters (always), a
    product lower bound on another pair (for about half of the seeds) and a
    divisibility clause (for about 60 % of the seeds with a list starting
    at 1)."""
    vals = []
    stream = 0
    total = 1
    while total < target_raw and len(vals) < 16:
        rem = target_raw / total
        if rem < 1.5 and len(vals) >= 3:
            break
        uu = float(uniform01(seed, 40 + stream, np.arange(2))[0])
        k = int(min(max_radix, max(2, round(2 + uu * (max_radix - 2)))))
        if rem < k * 1.5 or len(vals) == 15:
            k = int(max(2, min(31, round(rem))))
        style = float(uniform01(seed, 80 + stream, np.arange(1))[0])
        if style < 0.5 and k <= 20:
            vals.append(tuple(1 << e for e in range(k)))
        elif style < 0.8:
            vals.append(tuple(range(1, k + 1)))
        else:
            vals.append(tuple(range(k)))
        total *= k
        stream += 1
    n = len(vals)
    cu = uniform01(seed, 90, np.arange(16))
    clauses = []
    if n >= 2:
        i = int(cu[0] * n)
        j = (i + 1 + int(cu[1] * (n - 1))) % n
        lo = min(vals[i]) * min(vals[j])
        hi = max(vals[i]) * max(vals[j])
        if hi > lo:
            frac = 0.4 + 0.4 * cu[2]
            bound = int(round(max(lo, 1) * (hi / max(lo, 1)) ** frac))
            clauses.append(Clause("prod_le", tuple(sorted((i, j))), (), max(bound, lo)))
        divs = [k for k in range(n) if vals[k][0] == 1 and len(vals[k]) > 1]
        if divs and cu[3] < 0.6:
            d = divs[int(cu[4] * len(divs))]
            a = (d + 1 + int(cu[5] * (n - 1))) % n
            if a != d:
                clauses.append(Clause("divides", (a,), (d,)))
        if n >= 3 and cu[6] < 0.5:
            i2 = int(cu[7] * n)
            j2 = (i2 + 1 + int(cu[8] * (n - 1))) % n
            lo2 = max(min(vals[i2]), 1) * max(min(vals[j2]), 1)
            hi2 = max(max(vals[i2]), 1) * max(max(vals[j2]), 1)
            if hi2 > lo2:
                bound = int(round(lo2 * (hi2 / lo2) ** (0.05 + 0.25 * cu[9])))
                if bound > lo2:
                    clauses.append(Clause("prod_ge", tuple(sorted((i2, j2))), (), bound))
    return SpaceSpec(f"sized_{seed}_{target_raw}", tuple(f"p{i}" for i in range(n)),
                     tuple(vals), tuple(clauses))


def tiny_spaces(count: int, seed0: int = 1000, max_raw: int = 5000):
    """Small random spaces (<= ``max_raw`` raw points) for brute-force checks."""
    out = []
    s = seed0
    while len(out) < count:
        n = 1 + int(uniform01(s, 7, np.arange(1))[0] * 5)
        sp = random_space(s, n, max_radix=7, n_clauses=int(uniform01(s, 8, np.arange(1))[0] * 3))
        if sp.n_raw <= max_raw:
            out.append(sp)
        s += 1
    return out


# --------------------------------------------------------------------------
# batched workloads (many spaces of uneven size) and a device-side runtime
# model for them
# --------------------------------------------------------------------------

def _loguniform(seed: int, stream: int, count: int, lo: float, hi: float) -> np.ndarray:
    u = uniform01(seed, stream, np.arange(count))
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


# Valid-size targets: templates are rejection-sampled until their number of
# VALID configurations lies within +-20 % of a log-uniform target.  Counting
# valid configurations is the method's own arithmetic (the constraint mask),
# which this module does not hold, so the accepted candidates are read from a
# table (candidate index and raw-size target per template) that
# tests/golden/make_templates.py writes with the CPU oracle; that script
# also records each template's valid count, which a test re-checks.
TEMPLATE_TABLE = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                              "tests", "golden", "templates.json")
VALID_TOL = 0.20

# (seed, count of random templates, log-uniform valid-size range) per family
TEMPLATE_FAMILIES = {
    "batch": (7, 23, 1e3, 5e6),    # + the paper's three spaces = 26 templates
    "sweep": (11, 64, 1e4, 2e6),
}


def valid_targets(family: str) -> np.ndarray:
    """The valid-size target of every random template of ``family``:
    log-uniform over the family's range, drawn stratified (one target per
    equal slice of the log range, slices assigned to templates in a seeded
    random order), so that the batch's total size stays near its expected
    value instead of following the heavy tail of independent draws."""
    seed, count, lo, hi = TEMPLATE_FAMILIES[family]
    order = np.argsort(uniform01(seed, 1, np.arange(count)), kind="stable")
    u = (order + uniform01(seed, 2, np.arange(count))) / count
    return np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))


def template_candidate(family: str, t: int, k: int, target_raw: int) -> SpaceSpec:
    """Candidate k of template t of ``family``, with about target_raw raw points."""
    seed = TEMPLATE_FAMILIES[family][0]
    return sized_random_space(seed * 100000 + t * 1000 + k, int(target_raw))


def _template_table():
    with open(TEMPLATE_TABLE) as fh:
        return json.load(fh)


def family_templates(family: str, prefix: str):
    """The accepted random templates of ``family`` (see TEMPLATE_TABLE)."""
    rows = _template_table()[family]
    out = []
    for t, row in enumerate(rows):
        sp = template_candidate(family, t, row["k"], row["raw_target"])
        out.append(SpaceSpec(f"{prefix}_{t}", sp.names, sp.values, sp.clauses))
    return out


def batch_templates():
    """The paper's convolution, GEMM and PnPoly spaces plus 23 seeded random
    templates whose valid sizes are log-uniform in [1e3, 5e6] (+-20 %)."""
    return [conv_space(), gemm_space(), pnpoly_space()] + family_templates("batch", "template")


FAIL_LEVELS = (0.03, 0.30, 0.70)


def batch_workload(n_seeds: int = 9, seed_base: int = 0):
    """(space, seed, fail_frac) for every template x fitness seed (26 x 9 =
    234 spaces); the failure fraction cycles over 3 %, 30 % and 70 % by
    template.  ``seed_base`` shifts every fitness seed (another draw of the
    same templates)."""
    jobs = []
    for t, sp in enumerate(batch_templates()):
        for s in range(n_seeds):
            jobs.append((sp, seed_base + 100 * t + s + 1, FAIL_LEVELS[t % 3]))
    return jobs


def sweep_spaces():
    """64 seeded random spaces whose valid sizes are log-uniform in [1e4, 2e6]
    (+-20 %)."""
    return family_templates("sweep", "sweep")


def _mix64_t(z):
    """SplitMix64 finaliser on int64 tensors (two's-complement wrap-around,
    logical shifts emulated with masks)."""
    import torch
    m30 = (1 << 34) - 1
    m27 = (1 << 37) - 1
    m31 = (1 << 33) - 1
    c1 = torch.tensor(0xBF58476D1CE4E5B9 - (1 << 64), dtype=torch.int64, device=z.device)
    c2 = torch.tensor(0x94D049BB133111EB - (1 << 64), dtype=torch.int64, device=z.device)
    z = z ^ ((z >> 30) & m30)
    z = z * c1
    z = z ^ ((z >> 27) & m27)
    z = z * c2
    return z ^ ((z >> 31) & m31)


def _s64(v: int) -> int:
    v &= _M64
    return v - (1 << 64) if v >= (1 << 63) else v


def uniform01_torch(seed: int, stream: int, n: int, device):
    """The counter-based U[0,1) stream of ``uniform01`` evaluated on a device."""
    import torch
    idx = torch.arange(1, n + 1, dtype=torch.int64, device=device)
    gamma = torch.tensor(_s64(_GAMMA), dtype=torch.int64, device=device)
    z = torch.tensor(_s64(_base(seed, stream)), dtype=torch.int64, device=device) + idx * gamma
    h = _mix64_t(z)
    return ((h >> 11) & ((1 << 53) - 1)).to(torch.float64) * (1.0 / 9007199254740992.0)


def runtimes_torch(spec: SpaceSpec, seed: int, fail_frac: float = 0.03, noise_sd: float = 0.05,
                   device="cuda", n_bumps: int = 3):
    """``runtimes`` evaluated with torch on ``device`` (float64).  Same model
    and same counter streams; transcendental functions may differ from
    numpy's in the last bits, so use one or the other consistently."""
    import torch
    n = spec.n_params
    shape = spec.radix
    z = [torch.as_tensor(_coordinate(v), device=device) for v in spec.values]
    a = _uniform_n(seed, 1, n, 0.2, 1.0)
    m = _uniform_n(seed, 2, n, -0.6, 0.6)
    bij = _uniform_n(seed, 3, n * n, -0.15, 0.15).reshape(n, n)
    h = _uniform_n(seed, 4, n_bumps, 0.3, 0.8)
    sig = _uniform_n(seed, 5, n_bumps, 0.15, 0.35)
    mu = _uniform_n(seed, 6, n_bumps * n, -1.0, 1.0).reshape(n_bumps, n)

    def axis(i, vec):
        s = [1] * n
        s[i] = vec.shape[0]
        return vec.reshape(s)

    g = torch.zeros(shape, dtype=torch.float64, device=device)
    for i in range(n):
        g += axis(i, float(a[i]) * (z[i] - float(m[i])) ** 2)
    for i in range(n):
        for j in range(i + 1, n):
            g += float(bij[i, j]) * axis(i, z[i] - float(m[i])) * axis(j, z[j] - float(m[j]))
    for k in range(n_bumps):
        bump = torch.ones(shape, dtype=torch.float64, device=device)
        for i in range(n):
            bump = bump * axis(i, torch.exp(-((z[i] - float(mu[k, i])) ** 2) /
                                            (2.0 * float(sig[k]) ** 2)))
        g -= float(h[k]) * bump
    g = g.reshape(-1)
    R = spec.n_raw
    u1 = uniform01_torch(seed, 101, R, device)
    u2 = uniform01_torch(seed, 102, R, device)
    eps = noise_sd * torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)
    rt = torch.exp(1.0 + g + eps)
    if fail_frac > 0:
        rt[uniform01_torch(seed, 103, R, device) < fail_frac] = FAIL_RUNTIME
    return rt
