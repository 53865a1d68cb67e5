"""CPU-side checks of the C-ABI library: it builds for sm_103a, loads without a
GPU, exports every entry point include/fc.h declares, and its host-only
functions agree with the oracle."""
import ctypes
import math

import pytest

from oracle import dense
from paper_2101_06192_gb300 import build, fc


def test_library_builds_and_exports_declared_symbols():
    path = build.build()
    L = ctypes.CDLL(path)
    declared = fc.declared_symbols()
    assert "fc_sample_usts" in declared and "fc_build_augmented" in declared
    for name in declared:
        assert hasattr(L, name), name


@pytest.mark.parametrize("eps,delta,kappa,m", [(0.1, 0.1, 0.5, 60), (0.05, 1e-3, 0.3, 10**6),
                                               (0.3, 0.5, 0.9, 17), (0.4, 1 / 58000, 0.5, 214078)])
def test_tau_for_matches_oracle(eps, delta, kappa, m):
    assert fc.tau_for(eps, delta, kappa, m) == dense.tau_for(eps, delta, kappa, m)


def test_tau_for_rejects_bad_arguments():
    assert fc.tau_for(0.0, 0.1, 0.5, 10) == -1
    assert fc.tau_for(0.1, 1.0, 0.5, 10) == -1
    assert fc.tau_for(0.1, 0.1, 0.5, 0) == -1


def test_status_strings():
    L = fc.lib()
    for s in range(7):
        assert L.fc_status_str(s)
    assert L.fc_status_str(99) == b"unknown status"


def test_null_graph_arguments_rejected_without_gpu():
    L = fc.lib()
    assert L.fc_graph_info(None, None, None, None, None) == fc.FC_EINVAL
    assert L.fc_sample_usts(None, 1, 1, 0, None, None, None, 0, None, None) == fc.FC_EINVAL
    assert L.fc_set_sampler_shape(None, 32, 0, 0, 0) == fc.FC_EINVAL
    L.fc_destroy(None)


def test_null_arguments_of_the_next_rows_rejected_without_gpu():
    # Rao-Blackwellised accumulation, tree roots, root counts and group
    # closeness check their arguments before touching the device
    L = fc.lib()
    assert L.fc_rb_accumulate(None, 0, None, 1, None, None) == fc.FC_EINVAL
    assert L.fc_rb_diag(None, 10, 1, None, None) == fc.FC_EINVAL
    assert L.fc_tree_roots(None, 10, 1, None, None, None) == fc.FC_EINVAL
    assert L.fc_root_counts(None, 10, 1, None, 1, None, None) == fc.FC_EINVAL
    assert L.fc_group_closeness(None, 0, 1, 1e-12, None, None, None) == fc.FC_EINVAL
    assert L.fc_farness_from_diag(None, None, None, None, None) == fc.FC_EINVAL
