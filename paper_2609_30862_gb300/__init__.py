"""GB300-native QIEO generation loop for the 0/1 knapsack.

The compute path is the CUDA library built from csrc/ (C ABI declared in include/qieo.h);
`paper_2609_30862_gb300.qieo` is its thin ctypes binding and `workload` draws the seeded
synthetic instances. Nothing is imported here so that the workload module stays usable
without the CUDA library.
"""
