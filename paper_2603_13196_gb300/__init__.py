"""GB300-native batched likelihood of the region-partitioned global-21cm
foreground model (arXiv 2603.13196).

The compute lives in the C-ABI library libfg21 (include/fg21.h, sources in
csrc/, built by build.py); `fg21` is its Python binding, `inputs` the seeded
synthetic workload generator, and `ns` a batched slice-sampling nested-sampling
driver that feeds the library's serving loop.
"""
