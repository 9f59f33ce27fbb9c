"""GB300-native two-site DMRG effective-Hamiltonian library (Python binding).

The compute path is the CUDA shared library ``libtnh.so`` built from
``csrc/`` for sm_103a; ``tnh`` marshals arguments to its C ABI. Importing
this package does not load the library; ``tnh.lib()`` does, and fails
loudly when it has not been built.
"""
