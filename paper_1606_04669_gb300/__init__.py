"""Parallel Space Saving (Cafaro et al., arXiv:1606.04669) on one GB300.

The hot path (per-block Space Saving, the combine tree of Algorithm 2 and
the k-majority query) runs in the sm_103a kernels of libpss (csrc/), behind
the C ABI of include/pss.h, and so does the Frequent (Misra–Gries) summary
with its merge on the same blocks and tree.  This package is its thin
Python binding.
"""
from .pss import (  # noqa: F401
    Batch, PSS_EDEVICE, PSS_EINVAL, PSS_EMISMATCH, PSS_ENOMEM, PSS_ERANGE, PSS_MAX_K, PSS_MAX_K_RESIDENT, PSS_OK,
    Exported,
    PssError, Server, Summary, Tree, gen_zipf, lib_path, load, merge, profile_enable, profile_read, strerror,
    plan_blocks, plan_cta_shape, plan_kernel, set_round_kmax, set_warp_kmax, summarize, summarize_host, summarize_tree, exact_counts,
    QUERY_CANDIDATES, QUERY_GUARANTEED, import_summary, set_host_direct,
    KIND_SPACE_SAVING, KIND_FREQUENT, frequent, frequent_host, frequent_tree, estimate_skew,
    skew_of_pairs)
