"""B300-native molecular transition form factors (Cartesian Gaussian basis).

The compute path is the CUDA library ``libscff.so`` behind the C ABI in
``include/scff.h``; :mod:`paper_2512_18010_b300.scff` is its Python binding
and :mod:`paper_2512_18010_b300.workloads` draws seeded synthetic inputs.
"""
__all__ = ["scff", "workloads", "build"]
