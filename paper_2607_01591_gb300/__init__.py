"""GB300-native (sm_103a) planar flat-source Method of Characteristics transport sweep.

The CUDA library (paper_2607_01591_gb300/_lib/libmoc_gb300.so, C ABI in include/moc_gb300.h)
does all transport work; `moc.Moc` is its thin Python binding and `workloads` makes seeded
synthetic meshes and cross sections.
"""
__all__ = ["build", "moc", "workloads"]
