"""B300-native explicit 1D3V electrostatic PIC-MCC particle step.

``paper_2609_17151_b300.pic`` is the thin Python binding of the C-ABI library
``libpic1d3v.so`` (CUDA, sm_103a); ``paper_2609_17151_b300.workloads`` builds
the seeded synthetic inputs.  Importing the package itself loads nothing.
"""
