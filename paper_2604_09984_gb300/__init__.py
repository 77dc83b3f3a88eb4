"""GB300-native implicit unsteady UGKS on moving / overset meshes.

The compute path is the CUDA library ``libugks.so`` (sources in ``csrc/``,
C ABI in ``include/ugks.h``) reached through the ctypes binding
``paper_2604_09984_gb300.ugks``; ``workloads`` builds the seeded synthetic
configurations.  Importing this package does not load the library.
"""
