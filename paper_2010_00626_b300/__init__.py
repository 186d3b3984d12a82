"""B300-native kappa-cycle multigrid (Avnat & Yavneh, arXiv 2010.00626).

``paper_2010_00626_b300.kcycle`` binds the C ABI of ``libkcycle.so`` (include/kcycle.h);
``paper_2010_00626_b300.inputs`` holds the seeded synthetic workloads. Nothing heavy is
imported here, so the input generators can be used without the CUDA library.
"""
