// hydro_sums.cuh -- exact per-sub-grid sums of 512 doubles (the first pass of
// the grid totals and of the diagnostics sums).
//
// One warp sums the 512 values of one (sub-grid, quantity): it finds their
// largest binary exponent E (zero and subnormals count as exponent 1) and adds
// the significands as signed 128-bit fixed-point numbers with 63 guard bits
// below the last bit of a value of exponent E (values more than 63 binades
// below E keep their leading bits only).  Integer sums do not depend on the
// order, so any split of the 512 values over the lanes gives the same result.
// Output: 3 words per (sub-grid, quantity): the low and high word of the sum
// and E (0x7ff when a value is not finite).
#pragma once
#include <cuda_runtime.h>

namespace hydro {

constexpr int PARTIAL_WORDS = 3;

// ld(r) returns this lane's value r of 16 (the lanes together cover the 512);
// lane 0 writes the three words to out.
template <class Load>
__device__ __forceinline__ void warp_exact_sum(const Load& ld, unsigned long long* out) {
  const int lane = threadIdx.x & 31;
  unsigned long long b[16];
  unsigned emax = 1;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    b[r] = (unsigned long long)__double_as_longlong(ld(r));
    const unsigned e = (unsigned)(b[r] >> 52) & 0x7ffu;
    emax = e > emax ? e : emax;
  }
  emax = __reduce_max_sync(0xffffffffu, emax);
  __int128 acc = 0;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    unsigned e = (unsigned)(b[r] >> 52) & 0x7ffu;
    unsigned long long m = b[r] & 0x000fffffffffffffull;
    if (e)
      m |= 0x0010000000000000ull;
    else
      e = 1;
    const int sh = 63 - (int)(emax - e);  // bit position of the significand's last bit
    unsigned __int128 F;
    if (sh >= 0)
      F = (unsigned __int128)m << sh;
    else
      F = sh > -64 ? (unsigned __int128)(m >> (-sh)) : (unsigned __int128)0;
    acc += (b[r] >> 63) ? -(__int128)F : (__int128)F;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long lo = __shfl_down_sync(0xffffffffu, (unsigned long long)acc, o);
    const unsigned long long hi = __shfl_down_sync(0xffffffffu, (unsigned long long)((unsigned __int128)acc >> 64), o);
    acc += (__int128)(((unsigned __int128)hi << 64) | lo);
  }
  if (lane == 0) {
    out[0] = (unsigned long long)acc;
    out[1] = (unsigned long long)((unsigned __int128)acc >> 64);
    out[2] = emax;
  }
}

}  // namespace hydro
