"""GB300 (sm_103a) CKKS hot path: negacyclic NTT over RNS limbs, dyadic
product, Mul, Relin and RS behind the C ABI of include/he.h, after
"Accelerating Encrypted Computing on Intel GPUs" (arXiv 2109.14704).

Modules: ``he`` (binding of libhe.so), ``build`` (nvcc build), ``synth``
(seeded input generators), ``autotune`` (kernel-shape search), ``serving``
(continuous-batching request loop)."""
