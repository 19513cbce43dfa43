// gp_check.cuh -- index checks of the bounds-checked debug build (-DGP_CHECK).
//
// GP_IN_RANGE(site, i, n) guards an access: in the checked build it is true
// when 0 <= i < n, and otherwise records the first failure of the translation
// unit, (site << 40) | index, in a device word and is false, so that the
// caller skips the access instead of touching memory out of bounds.  In the
// default build it is the constant true and the checks compile away.
// GP_CHECK_READER(name) defines, in the checked build, a host function that
// reads and clears the word of its own translation unit (each .cu file has its
// own copy: the variable has internal linkage).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#ifdef GP_CHECK
namespace gp {
namespace check {
static __device__ unsigned long long g_first_failure = 0ull;

__device__ __forceinline__ bool in_range(int site, long long i, long long n) {
  if (i >= 0 && i < n) return true;
  const unsigned long long word = ((unsigned long long)site << 40) | ((unsigned long long)i & ((1ull << 40) - 1ull));
  atomicCAS(&g_first_failure, 0ull, word);
  return false;
}
}  // namespace check
}  // namespace gp
#define GP_IN_RANGE(site, i, n) (::gp::check::in_range((site), (long long)(i), (long long)(n)))
#define GP_CHECK_READER(name)                                                   \
  unsigned long long name() {                                                   \
    unsigned long long v = 0ull, z = 0ull;                                      \
    if (cudaMemcpyFromSymbol(&v, ::gp::check::g_first_failure, sizeof(v)) != cudaSuccess) { \
      cudaGetLastError();                                                       \
      return 0ull;                                                              \
    }                                                                           \
    if (v) cudaMemcpyToSymbol(::gp::check::g_first_failure, &z, sizeof(z));     \
    return v;                                                                   \
  }
#else
#define GP_IN_RANGE(site, i, n) true
#define GP_CHECK_READER(name)
#endif
