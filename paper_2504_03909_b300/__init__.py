"""B300-native Paillier hot path of vertical secure federated XGBoost.

Submodules:
  paillier  - torch-tensor API over the C ABI (encode/encrypt/aggregate/decrypt)
  native    - ctypes binding of include/paillier.h
  synth     - seeded synthetic inputs (shapes of the paper's workloads)
  build     - in-tree nvcc build of libpaillier_b300.so

Importing the package does not load the native library; the first call that
needs it does, and fails loudly if it has not been built.
"""
