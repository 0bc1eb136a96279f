// The synthetic Hamiltonian's element generator (Eq. (ham) of Sec. II.A made
// index-addressable): Philox4x32-10 (Salmon et al., SC'11), Box-Muller, then the
// antisymmetrised, Hermitised element.  Shared by every kernel that writes integrals.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

typedef double2 cplx;  // (re, im)

__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

// A[idx]: complex standard normal via Box-Muller of two 53-bit uniforms.
__device__ __forceinline__ cplx gauss_a(uint64_t idx, uint64_t seed) {
  uint32_t c[4] = {uint32_t(idx), uint32_t(idx >> 32), 0u, 0u};
  philox10(c, uint32_t(seed), uint32_t(seed >> 32));
  const uint64_t a = ((uint64_t(c[1]) << 32) | c[0]) >> 11;
  const uint64_t b = ((uint64_t(c[3]) << 32) | c[2]) >> 11;
  const double u1 = (double(a) + 0.5) * 0x1p-53;
  const double u2 = (double(b) + 0.5) * 0x1p-53;
  const double rad = sqrt(-2.0 * log(u1));
  double s, co;
  sincospi(2.0 * u2, &s, &co);
  return make_double2(rad * co, rad * s);
}

// V_pqrs = 1/2 [ (A_pqrs - A_qprs - A_pqsr + A_qpsr) + conj(A_rspq - A_srpq - A_rsqp + A_srqp) ]
__device__ __forceinline__ cplx v_element(uint64_t p, uint64_t q, uint64_t r, uint64_t s, uint64_t n, uint64_t seed) {
  auto I = [n](uint64_t a, uint64_t b, uint64_t c, uint64_t d) { return ((a * n + b) * n + c) * n + d; };
  const cplx x0 = gauss_a(I(p, q, r, s), seed), x1 = gauss_a(I(q, p, r, s), seed);
  const cplx x2 = gauss_a(I(p, q, s, r), seed), x3 = gauss_a(I(q, p, s, r), seed);
  const cplx y0 = gauss_a(I(r, s, p, q), seed), y1 = gauss_a(I(s, r, p, q), seed);
  const cplx y2 = gauss_a(I(r, s, q, p), seed), y3 = gauss_a(I(s, r, q, p), seed);
  const double xr = x0.x - x1.x - x2.x + x3.x, xi = x0.y - x1.y - x2.y + x3.y;
  const double yr = y0.x - y1.x - y2.x + y3.x, yi = y0.y - y1.y - y2.y + y3.y;
  return make_double2(0.5 * (xr + yr), 0.5 * (xi - yi));
}
