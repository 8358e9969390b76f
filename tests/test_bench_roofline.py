"""bench.py's roofline denominators (host logic, no GPU): which kernel
categories are bounded by memory traffic, and the FP32 ALU peak derived from
the SM count and the sampled clock."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


class _Props:
    multi_processor_count = 148


class _Cuda:
    @staticmethod
    def get_device_properties(i):
        return _Props()


class _Torch:
    cuda = _Cuda()


def test_sweeps_and_vector_kernels_are_memory_bound_factor_kernels_count_flops():
    for k in ("apply_leaf_up", "apply_group_down", "spmv", "pcg_vector", "extend_add",
              "assemble_fd", "band_inverse"):
        assert bench.hbm_bound(k)
    for k in ("skel", "partial_chol", "leaf_elim", "precond_scale", "precond_diag"):
        assert not bench.hbm_bound(k)


def test_fp32_peak_from_the_device_sm_count_and_the_sampled_clock():
    peak, kind = bench.alu_peak_nominal("fp32", _Torch(), 1500)
    assert abs(peak - 148 * 128 * 2 * 1.5e9 / 1e12) < 1e-9
    assert "148 SMs" in kind and "1500 MHz" in kind
    # no clock sample: the maximum SM clock of GB300
    peak, _ = bench.alu_peak_nominal("fp32", _Torch(), None)
    assert abs(peak - 148 * 128 * 2 * 2.07e9 / 1e12) < 1e-9
    assert bench.alu_peak_nominal("fp64")[0] == 1.25
