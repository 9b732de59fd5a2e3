"""Named synthetic workloads shaped like the paper's models (Sec. 4, Tables 1-3).

Each workload bundles a medium generator, the frequencies, the sources and
the solver tolerance.  Names say what the workload is and its size.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import media, sources


@dataclass
class Workload:
    name: str
    n: int
    h: float
    freqs_hz: tuple
    make_medium: object
    make_sources: object          # () -> (M6 array (k,6), xs array (k,3))
    tol: float
    precision: str                # "fp64" or "mixed"
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def medium(self):
        return self.make_medium()

    def sources(self):
        return self.make_sources()


def _centre(n, h):
    c = (n - 1) / 2.0 * h
    return np.array([c, c, c])


def _inclusion_sources():
    return sources.explosion()[None, :], _centre(16, 10.0)[None, :]


def _layers_sources():
    return sources.double_couple_12()[None, :], np.array([[315.0, 315.0, 400.0]])


def _grf_sources():
    rng = np.random.default_rng(media.BASE_SEED + 33)
    M = sources.random_moment_tensors(8, rng)
    xs = np.repeat(_centre(128, 8.0)[None, :], 8, axis=0)
    return M, xs


def _table2_sources():
    return sources.double_couple_13()[None, :], _centre(96, 10.0)[None, :]


def _tti_sources():
    M = np.stack([sources.explosion(1.0 / np.sqrt(3.0)), sources.clvd(),
                  sources.double_couple_12(), sources.double_couple_13()])
    xs = np.repeat(_centre(256, 5.0)[None, :], 4, axis=0)
    return M, xs


WORKLOADS = {
    # plain FP64 single solve, 16^3, VTI cube inclusion, explosion at the centre
    "inclusion16_fp64": Workload(
        "inclusion16_fp64", 16, 10.0, (10.0,),
        lambda: media.inclusion_medium(16, 10.0), _inclusion_sources, 1e-10, "fp64",
        notes="16^3, dx=10 m, 10 Hz, VTI 6^3 cube (eps=.1, delta=.05, gamma=.08, +5% rho), M=I"),
    # plain vs mixed, 64^3 three VTI layers, strike-slip DC, 5/15/30 Hz
    "layers64": Workload(
        "layers64", 64, 10.0, (5.0, 15.0, 30.0),
        lambda: media.layered_vti_medium(64, 10.0), _layers_sources, 1e-6, "mixed",
        notes="64^3, dx=10 m, 3 VTI layers, DC M12 at (315,315,400) m"),
    # batched 128^3 GRF orthorhombic, 32 frequencies x 8 moment tensors
    "grf128_batched": Workload(
        "grf128_batched", 128, 8.0, tuple(np.linspace(2.0, 40.0, 32)),
        lambda: media.grf_orthorhombic_medium(128, 8.0), _grf_sources, 1e-6, "mixed",
        notes="128^3, dx=8 m, 5% GRF orthorhombic contrast (L=40 m), 32 freqs 2-40 Hz x 8 random MTs"),
    # adjoint workload, 96^3 Table-2 layers + 3% GRF, dip-slip DC
    "table2_96_adjoint": Workload(
        "table2_96_adjoint", 96, 10.0, tuple(4.0 * (k + 1) for k in range(8)),
        lambda: media.table2_layers_medium(96, 10.0), _table2_sources, 1e-6, "mixed",
        notes="96^3, dx=10 m, Table 2 layers + 3% GRF, DC M13, 256 surface receivers"),
    # large batched mixed 256^3 TTI layer, 16 frequencies x 4 sources
    "tti256_batched": Workload(
        "tti256_batched", 256, 5.0, tuple(np.linspace(5.0, 60.0, 16)),
        lambda: media.tti_layer_medium(256, 5.0), _tti_sources, 1e-6, "mixed",
        notes="256^3, dx=5 m, TTI layer (tilt 30 deg), 16 freqs x 4 sources"),
}


def get_workload(name):
    return WORKLOADS[name]
