// Bounds-checked builds (compiled with -DTF_BOUNDS_CHECK, library libtf_checked.so).
//
// Every global-memory access of the product kernels goes through TF_IN(site, off, ext):
// in a normal build it is the constant true; in a checked build it tests 0 <= off < ext
// (the offset within the column's buffer and that buffer's extent) and, on a violation,
// records the first offending site, offset and extent in a per-translation-unit device
// word and returns false, so the caller skips the access instead of faulting.  The host
// reads and clears the records with tf_debug_oob().
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tfk {

struct OobRecord {
  unsigned int hit;
  int site;
  long long off;
  long long ext;
};

// Sites (which access of which kernel); generic-engine kernels add 100.
enum OobSite {
  kSiteR2cSrc = 1, kSiteR2cScale = 2, kSiteR2cDst = 3,
  kSiteC2rSrc = 4, kSiteC2rDst = 5, kSiteC2rScale = 6,
  kSiteFwdZ = 7, kSiteFwdSpec = 8, kSiteFwdS = 9,
  kSiteAdjZ = 10, kSiteAdjSpec = 11, kSiteAdjU = 12,
  kSiteSmem = 50
};

__device__ __forceinline__ bool oob_check(OobRecord* rec, int site, long long off, long long ext) {
  if (off >= 0 && off < ext) return true;
  if (atomicCAS(&rec->hit, 0u, 1u) == 0u) {
    rec->site = site;
    rec->off = off;
    rec->ext = ext;
  }
  return false;
}

}  // namespace tfk

#ifdef TF_BOUNDS_CHECK
// Each translation unit that includes this header gets its own record.
static __device__ tfk::OobRecord g_tf_oob;
#define TF_IN(site, off, ext) (tfk::oob_check(&g_tf_oob, (site), (long long)(off), (long long)(ext)))
#else
#define TF_IN(site, off, ext) (true)
#endif

// Host accessor for this translation unit's record (defined once per TU by
// TF_DEFINE_OOB_READER); returns false when the build is not checked.
#ifdef TF_BOUNDS_CHECK
#define TF_DEFINE_OOB_READER(name)                                              \
  bool name(tfk::OobRecord* out, bool clear) {                                   \
    if (cudaMemcpyFromSymbol(out, g_tf_oob, sizeof(*out)) != cudaSuccess) return false; \
    if (clear) {                                                                 \
      tfk::OobRecord z{0u, 0, 0, 0};                                             \
      cudaMemcpyToSymbol(g_tf_oob, &z, sizeof(z));                               \
    }                                                                            \
    return true;                                                                 \
  }
#else
#define TF_DEFINE_OOB_READER(name)                                              \
  bool name(tfk::OobRecord* out, bool) {                                         \
    *out = tfk::OobRecord{0u, 0, 0, 0};                                          \
    return false;                                                                \
  }
#endif
