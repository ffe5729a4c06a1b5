"""GB300-native (sm_103a) implementation of the FSZ compress/decompress hot path.

``fsz`` binds the C ABI of the CUDA library (include/fsz.h); ``inputs`` holds the
seeded synthetic workload generators.
"""
from . import fsz  # noqa: F401
from .fsz import (EB_ABS, EB_REL, FszError, Workspace, compress, decompress,  # noqa: F401
                  fsz_batch_workspace_bytes, fsz_check, fsz_check_batched, fsz_compress,
                  fsz_compress_batched, fsz_compress_bound, fsz_compress_encode,
                  fsz_compress_prepare, fsz_decompress, fsz_decompress_batched, fsz_read_header,
                  fsz_set_test_hooks, fsz_version, fsz_workspace_bytes, lib)

__all__ = ["fsz", "compress", "decompress", "lib"]
