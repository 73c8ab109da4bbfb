"""TensorACO on GB300: the per-iteration ant colony path as sm_103a CUDA kernels
behind a C ABI (include/tensoraco.h); this package is the thin Python binding."""
