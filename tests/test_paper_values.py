"""Values the paper prints, kept as a golden fixture with citations."""
import json
import os

from oracle import rihv_oracle as O
from paper_1904_04884_gb300 import workloads

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


def test_storage_arithmetic():
    assert O.dense_bytes(1) == GOLD["dense_bytes_per_voxel"]["value"]
    assert O.coo_bytes(1) == GOLD["coo_bytes_per_nnz"]["value"]
    assert round(100 * O.coo_break_even_sparsity()) == GOLD["coo_break_even_sparsity_percent"]["value"]
    assert round(O.dense_bytes(1024 ** 3) / 2 ** 30) == GOLD["volume_1024cubed_GB"]["value"]


def test_shadow_density_example():
    g = GOLD["algae_shadow_density_percent"]
    n_s = g["inputs"]["cells_per_mL"] * 1e6          # per m^3
    depth, d = g["inputs"]["depth_m"], g["inputs"]["diameter_m"]
    area = 1e-6                                       # any area: s_d is intensive
    s = workloads.shadow_density(n_s * area * depth, depth, d, area)
    assert round(100 * s) == g["value"]


def test_turbulence_volume_size():
    g = GOLD["turbulence_voxels"]
    nx, ny, nz = g["shape"]
    assert abs(nx * ny * nz - g["value"]) / g["value"] < 0.02
    w = workloads.PAPER_TURBULENCE
    assert (w.nx, w.ny, w.nz) == (nx, ny, nz)
