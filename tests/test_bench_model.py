"""The bench's algorithmic-byte model (no GPU): the per-launch bytes of each kernel kind
for the 256^3 workload, written out from the array sizes they read and write, so a change
to the model or to a workload shows up here before it moves a roofline fraction."""

import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import bench  # noqa: E402
from paper_1707_09898_gb300 import workloads as W  # noqa: E402

N = 256
K = 512 // 2 + 1               # half spectrum
CELLS = N * N * N              # design cells (nzd = 256)
SPEC = 8 * N * N * K           # one complex64 half-spectrum volume of the design planes
TZ = N * (512 // 2 + 1) * K * 4  # one x/y-transformed tensor component over the design offsets
PLANE = 8 * 512 * K            # one y-spectrum plane


@pytest.fixture(scope="module")
def model():
    wl = W.config4(N)
    return (bench.alg_bytes(wl, (512, 512, 512), direct=True, fused=True),
            bench.alg_bytes(wl, (512, 512, 512), direct=True, fused=True, step_fused=True))


def test_main_kernels(model):
    ab, _ = model
    assert ab["x_forward"] == 4 * CELLS + SPEC                    # rho in, one spectrum out
    assert ab["yz_forward"] == SPEC + TZ + PLANE                  # spectra, zz tensor, target plane
    assert ab["zy_adjoint"] == 8 * N * K + TZ + SPEC              # source rows, tensor, design planes
    assert ab["x_inverse"] == SPEC + 8 * CELLS                    # spectra + rho in, G out


def test_fused_step_adds_gradient_in_and_rho_out(model):
    ab, abs_ = model
    assert abs_["x_forward"] - ab["x_forward"] == 8 * CELLS
    # without the fusion the update is a kernel of its own: rho and G in, rho out
    assert ab["other"] == 12 * CELLS and "other" not in abs_
    rest = ("x_forward", "other")
    assert {k: v for k, v in abs_.items() if k not in rest} == {k: v for k, v in ab.items() if k not in rest}


def test_stray_field_model():
    sf = bench.stray_field_bytes(W.config4(N), (512, 512, 512))
    T = (512 // 2 + 1) ** 2 * K * 4  # one folded tensor component
    assert sf["x_forward"] == 4 * CELLS + SPEC
    assert sf["z_pass"] == 8 * K * 512 * (N + 3 * N) + 3 * T   # M0 along z reaches xz, yz, zz
    assert sf["x_inverse"] == 3 * (SPEC + 4 * CELLS)


def test_step_total_is_about_a_gigabyte(model):
    _, abs_ = model
    big = abs_["x_forward"] + abs_["yz_forward"] + abs_["zy_adjoint"] + abs_["x_inverse"]
    assert 1.00e9 < big < 1.02e9
