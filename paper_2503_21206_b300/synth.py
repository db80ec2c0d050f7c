"""Seeded synthetic workloads shaped like the paper's datasets (Sec. 6.1).

The paper measures on DEEP (96-d), T2I, WIKI and LAION (768-d) at 100M and 1M
scale.  None of those datasets is available here, so these generators stand in
for them with the same dimensions and with controlled spectra.  Every array is
a pure function of its seed.  This module holds no search arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    """One benchmark / parity configuration."""
    name: str
    kind: str              # "mixture" | "powerlaw"
    n: int                 # base vectors
    d: int                 # dimension
    nq: int                # queries
    R: int                 # full-graph out-degree
    R_sub: int             # subgraph out-degree
    sample_ratio: float    # subgraph node sampling ratio (Sec. 4.1 (1))
    dp: int                # reduced dimension d'
    n_entry: int           # FES entry-set size
    k: int
    efs: tuple             # ef values swept
    metric: int            # 0 = squared L2, 1 = inner product
    n_comp: int = 0        # mixture components
    sigma: float = 0.0     # mixture spread
    power: float = 0.0     # per-dimension variance ~ i^-power before rotation
    unit_norm: bool = False
    seed: int = 0          # c: data 1000+c, queries 2000+c, graph/sample 3000+c, entries 4000+c
    reduced_dtypes: tuple = ("f32",)
    extra: dict = field(default_factory=dict)

    @property
    def data_seed(self):
        return 1000 + self.seed

    @property
    def query_seed(self):
        return 2000 + self.seed

    @property
    def graph_seed(self):
        return 3000 + self.seed

    @property
    def entry_seed(self):
        return 4000 + self.seed


# The workloads.  C1 is the small parity case; C2 is the plain FP32 1M x 96
# workload the benchmark times; C3-C5 are the precision, serving and
# memory-bounded shapes.
WORKLOADS = {
    "c1_mixture_20k_d96": Workload("c1_mixture_20k_d96", "mixture", 20_000, 96, 200, 32, 32, 0.25, 32, 256,
                                   10, (64,), 0, n_comp=100, sigma=0.3, seed=1),
    "c2_aniso_1m_d96": Workload("c2_aniso_1m_d96", "powerlaw", 1_000_000, 96, 10_000, 32, 32, 0.30, 32, 4096,
                                10, (32, 64, 128, 256), 0, power=0.8, unit_norm=True, seed=2),
    "c3_powerlaw_2m_d768": Workload("c3_powerlaw_2m_d768", "powerlaw", 2_000_000, 768, 10_000, 48, 48, 0.25, 128,
                                    4096, 10, (64, 128, 256), 1, power=1.0, unit_norm=True, seed=3,
                                    reduced_dtypes=("f32", "bf16", "fp8")),
    # 10,000 well-separated components: 32,768 entries (about 3 per component)
    # let fast entry selection land each query in its own component
    "c4_mixture_10m_d256": Workload("c4_mixture_10m_d256", "mixture", 10_000_000, 256, 10_000, 32, 32, 0.20, 64,
                                    32768, 10, tuple(range(32, 513, 32)), 0, n_comp=10_000, sigma=0.3, seed=4,
                                    reduced_dtypes=("bf16",)),
    "c5_powerlaw_25m_d768": Workload("c5_powerlaw_25m_d768", "powerlaw", 25_000_000, 768, 10_000, 32, 32, 0.15,
                                     128, 4096, 10, (64, 128, 192, 256, 384, 512), 1, power=1.0, unit_norm=True,
                                     seed=5, reduced_dtypes=("bf16",), extra={"device_base": True}),
}


def haar_rotation(d: int, rng: np.random.Generator) -> np.ndarray:
    """A Haar-distributed orthogonal matrix: QR of a Gaussian matrix (FP64)
    with the signs of R's diagonal moved into Q."""
    g = rng.standard_normal((d, d))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def _mixture(n: int, centres: np.ndarray, sigma: float, seed: int, chunk: int) -> np.ndarray:
    """Components and noise come from separate streams, so the first m rows
    do not depend on n (a smaller case is a prefix of a larger one)."""
    d = centres.shape[1]
    crng = np.random.default_rng([seed, 1])
    nrng = np.random.default_rng([seed, 2])
    out = np.empty((n, d), np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        comp = crng.integers(0, centres.shape[0], m)
        out[s:s + m] = centres[comp] + sigma * nrng.standard_normal((m, d))
    return out


def _powerlaw(n: int, d: int, power: float, rot: np.ndarray, unit: bool, rng: np.random.Generator,
              chunk: int) -> np.ndarray:
    std = np.arange(1, d + 1, dtype=np.float64) ** (-power / 2.0)
    out = np.empty((n, d), np.float32)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        z = rng.standard_normal((m, d)) * std[None, :]
        x = z @ rot.T
        if unit:
            x /= np.linalg.norm(x, axis=1, keepdims=True)
        out[s:s + m] = x
    return out


def generate(w: Workload, n: int | None = None, nq: int | None = None, chunk: int = 1 << 18):
    """(base n x d float32, queries nq x d float32) for workload ``w``.

    Mixture: centres ~ N(0, I), points = centre + sigma * N(0, I); queries from
    the same mixture.  Power law: z ~ N(0, diag(i^-power)), a seeded Haar
    rotation, optional unit normalisation; queries from the same law.
    ``n`` / ``nq`` override the sizes; a smaller case is a prefix of a larger one."""
    n = w.n if n is None else n
    nq = w.nq if nq is None else nq
    drng = np.random.default_rng(w.data_seed)
    qrng = np.random.default_rng(w.query_seed)
    if w.kind == "mixture":
        centres = drng.standard_normal((w.n_comp, w.d))
        base = _mixture(n, centres, w.sigma, w.data_seed, chunk)
        queries = _mixture(nq, centres, w.sigma, w.query_seed, chunk)
    elif w.kind == "powerlaw":
        rot = haar_rotation(w.d, drng)
        base = _powerlaw(n, w.d, w.power, rot, w.unit_norm, drng, chunk)
        queries = _powerlaw(nq, w.d, w.power, rot, w.unit_norm, qrng, chunk)
    else:
        raise ValueError(w.kind)
    return base, queries


def generate_base_on_device(w: Workload, n: int | None = None, device="cuda", chunk: int = 1 << 20):
    """A power-law base set drawn on the GPU, for workloads whose base set is
    too large to hold twice in host memory (the 25M x 768 one: 77 GB).  Same
    spectrum and the same rotation as ``generate`` (the rotation is the data
    generator's first draw); the normal samples come from torch's generator
    seeded with the data seed, so the rows differ from ``generate``'s but are
    a pure function of the seed.  Returns an n x d float32 CUDA tensor."""
    import torch
    if w.kind != "powerlaw":
        raise ValueError("generate_base_on_device draws power-law base sets")
    n = w.n if n is None else n
    rot = haar_rotation(w.d, np.random.default_rng(w.data_seed))
    dev = torch.device(device)
    g = torch.Generator(device=dev)
    g.manual_seed(w.data_seed)
    std = torch.arange(1, w.d + 1, dtype=torch.float64, device=dev).pow(-w.power / 2.0).float()
    rot_t = torch.from_numpy(rot.T.astype(np.float32)).to(dev)
    X = torch.empty((n, w.d), dtype=torch.float32, device=dev)
    for s in range(0, n, chunk):
        m = min(chunk, n - s)
        x = (torch.randn((m, w.d), generator=g, device=dev, dtype=torch.float32) * std) @ rot_t
        if w.unit_norm:
            x /= torch.linalg.vector_norm(x.double(), dim=1, keepdim=True).float()
        X[s:s + m] = x
    return X
