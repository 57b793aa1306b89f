"""All-pairs posterior stage of QuickProbs 2 on B300 (sm_103a).

The compute path is the CUDA library ``libqp.so`` (C ABI in include/qp.h);
this package is its thin ctypes binding.
"""
from .qp import (GUARD_BITS, QP_COMBINE, QP_F32_SCALED, QP_F64_PLAIN, QpError, Result,
                 Server, lib, make_family, make_params, qp_last_error, qp_consistency, qp_get_counter, qp_guide_tree, qp_pair_posteriors_static, qp_posteriors,
                 qp_posteriors_range, qp_set_option, qp_split_pairs,
                 qp_result_free, qp_server_cancel, qp_server_create,
                 qp_server_destroy, qp_server_get_stats, qp_server_poll, qp_server_submit, qp_version)

__all__ = [
    "GUARD_BITS", "QP_COMBINE", "QP_F32_SCALED", "QP_F64_PLAIN", "QpError", "Result", "Server",
    "lib", "make_family", "make_params", "qp_last_error", "qp_consistency", "qp_get_counter", "qp_guide_tree", "qp_pair_posteriors_static", "qp_posteriors",
    "qp_posteriors_range", "qp_set_option", "qp_split_pairs",
    "qp_result_free", "qp_server_cancel", "qp_server_create", "qp_server_destroy",
    "qp_server_get_stats", "qp_server_poll", "qp_server_submit", "qp_version",
]
