// Bounds checks of the MSP_CHECKED build of libmsp.
//
// Compiled with -DMSP_CHECKED (build.build(checked=True) writes
// libmsp_checked.so), the kernels test every global or shared index they
// form from data (an inner position from a bucket bound and a record
// number, a compacted element, a staged or sorted position) against the
// size of its array before the access.  A failed check records its site
// number in the check word of its translation unit and the access is
// skipped; no kernel traps.  After every solve the host reads and clears all
// check words, and a nonzero one fails the solve with MSP_ECUDA naming the
// site.  Without MSP_CHECKED every check is the constant true and compiles
// away.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

namespace msp {
#ifdef MSP_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif
// Reader of one translation unit's check word: returns the first failed
// site (0 = none) and clears the word.
using CheckReader = unsigned (*)();
void register_check_reader(CheckReader r);
// First failed site of any translation unit since the last call (0 = none);
// synchronises the device first.
unsigned take_check_sites();
}  // namespace msp

#ifdef MSP_CHECKED
namespace {
__device__ unsigned int g_msp_check_site;
__device__ __forceinline__ bool msp_in_bounds(uint64_t idx, uint64_t size, unsigned site) {
  if (idx < size) return true;
  atomicCAS(&g_msp_check_site, 0u, site);
  return false;
}
unsigned msp_take_check_word() {
  unsigned h = 0, z = 0;
  cudaMemcpyFromSymbol(&h, g_msp_check_site, sizeof(h));
  cudaMemcpyToSymbol(g_msp_check_site, &z, sizeof(z));
  return h;
}
struct MspCheckRegistration {
  MspCheckRegistration() { msp::register_check_reader(&msp_take_check_word); }
} g_msp_check_registration;
}  // namespace
#define MSP_IN_BOUNDS(idx, size, site) msp_in_bounds((idx), (size), (site))
#else
#define MSP_IN_BOUNDS(idx, size, site) true
#endif
