"""GB300-native sliding window sums and minimizers (arXiv 1811.10074).

The computation lives in a CUDA library with a C ABI (``include/sws.h``); ``binding`` is its
thin ctypes binding and ``synth`` the seeded input generators.  Importing the package does not
load the library; the first call does, and raises if it has not been built.
"""

from .binding import (Batch, Context, Server, SwsError, build_table, default_context, kmer_table,  # noqa: F401
                      kmers, minimizer_strands, minimizers, minimizers_batch, minimizers_count,
                      minimizers_from_keys, seed_hits, seed_lookup, sliding_sum, tune_sliding_sum)
