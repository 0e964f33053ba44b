"""GB300 (sm_103a) state-vector simulator core.

The product is the C-ABI library libsvgb300.so (include/sv.h), built in-tree by
paper_2604_03816_gb300.build; `paper_2604_03816_gb300.sv` is its Python binding.
Importing the package itself loads nothing, so that the build step can run first.
"""
