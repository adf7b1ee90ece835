"""GB300-native PC-stable skeleton learning with the G^2 test (Fast-BNS method).

The compute path is the CUDA library libfbn.so (include/fbn.h); ``fbn`` is its
thin ctypes binding with the same names.  Build with
``python -m paper_2212_04259_gb300.build``.
"""
from .fbn import (FbnError, Handle, fbn_create, fbn_set_stream, fbn_ci_test, fbn_ci_table,  # noqa: F401
                  fbn_learn_skeleton, fbn_learn_skeleton_batch, fbn_get_sepset, fbn_export_sepsets,
                  fbn_get_stats, fbn_orient_cpdag, fbn_last_error, fbn_destroy, fbn_ci_test_noalloc,
                  fbn_pairwise_counts, fbn_update_data, fbn_measure_unit_rates, fbn_autotune,
                  fbn_learn_skeleton_sharded, fbn_update_data_batch, lib, LIB_PATH, EXPORTS)
