// rewl_device.cuh -- device primitives of the REWL kernels: the Philox
// counter-based generator, the acceptance threshold lam = -ln u in 2^-32 fixed
// point, and lattice access for the two spin models.
#pragma once
#include <stdint.h>

#include "rewl_internal.h"

namespace rewl {

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds; each round
// multiplies counter words 0 and 2 by the two round constants (32x32 -> 64),
// mixes the high halves with words 1 and 3 and the key, and bumps the key by
// the Weyl constants.  Returns the four output words.
struct u32x4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ u32x4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                          uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Acceptance threshold of one trial: lam = -ln u with u = (k + 1) 2^-24 in
// binary32, returned as max(1, trunc(lam * 2^32)).  A trial whose ln g cost
// (ln g(E') - ln g(E), or the Eq. (1) sum, in 2^-32 units) is below the
// threshold is accepted: P(accept) = P(u < e^{-cost}) = min(1, g(E)/g(E')).
// Evaluation: u = 2^e m, m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(s) with
// s = (m-1)/(m+1) summed to s^9; e ln 2 with Cody & Waite's two-part ln 2
// (355/512 + ln2_lo) so that e * 355/512 is exact.  Every step is one IEEE
// binary32 operation rounded to nearest (explicit __f*_rn intrinsics, so the
// compiler neither fuses nor reorders), which makes the result identical on
// any IEEE-754 implementation of the same steps.
__device__ __forceinline__ long long lam_threshold(uint32_t k)
{
    const float kLn2Hi = 0.693359375f;                 // 355/512
    const float kLn2Lo = -2.12194440e-4f;              // ln 2 - 355/512
    const float kC9 = __uint_as_float(0x3de38e39u);    // 1/9 rounded
    const float kC7 = __uint_as_float(0x3e124925u);    // 1/7
    const float kC5 = __uint_as_float(0x3e4ccccdu);    // 1/5
    const float kC3 = __uint_as_float(0x3eaaaaabu);    // 1/3
    const float kSqrt2 = __uint_as_float(0x3fb504f3u); // 1.41421356f
    const float x = __uint2float_rn(k + 1u);           // exact: k + 1 <= 2^24
    const uint32_t bits = __float_as_uint(x);
    int e = (int)(bits >> 23) - 127;
    float m = __uint_as_float((bits & 0x007FFFFFu) | 0x3F800000u);
    if (m > kSqrt2) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float a = __fsub_rn(m, 1.0f);
    const float b = __fadd_rn(m, 1.0f);
    const float s = __fdiv_rn(a, b);
    const float z = __fmul_rn(s, s);
    float p = __fmaf_rn(z, kC9, kC7);
    p = __fmaf_rn(p, z, kC5);
    p = __fmaf_rn(p, z, kC3);
    p = __fmaf_rn(p, z, 1.0f);
    const float ln_m = __fmul_rn(__fadd_rn(s, s), p);
    const float ef = __int2float_rn(e - 24);
    const float t = __fmaf_rn(ef, kLn2Lo, ln_m);
    const float ln_u = __fmaf_rn(ef, kLn2Hi, t);
    const long long fix = __float2ll_rz(__fmul_rn(-ln_u, 4294967296.0f));
    return fix < 1 ? 1 : fix;
}

// uniform integer in [0, n)
__device__ __forceinline__ uint32_t scale_u32(uint32_t r, uint32_t n) { return __umulhi(r, n); }

// nearest integer to s / m, ties to even (m > 0)
__device__ __forceinline__ long long div_round_even(long long s, long long m)
{
    long long q = s / m, r = s % m;
    if (r < 0) {
        r += m;
        q -= 1;
    }
    if (2 * r > m || (2 * r == m && (q & 1))) q += 1;
    return q;
}

// ---------------------------------------------------------------------------
// lattices
// ---------------------------------------------------------------------------
// Site decomposition: y = floor(site / L) with one high multiply (exact for
// N L^2 < 2^32), periodic neighbours.
struct Site {
    int x, y, xl, xr, yu, yd;
};

__device__ __forceinline__ Site site_of(int site, int L, uint32_t magic_L)
{
    Site s;
    s.y = (int)__umulhi((uint32_t)site, magic_L);
    s.x = site - s.y * L;
    s.xl = s.x == 0 ? L - 1 : s.x - 1;
    s.xr = s.x == L - 1 ? 0 : s.x + 1;
    s.yu = s.y == 0 ? L - 1 : s.y - 1;
    s.yd = s.y == L - 1 ? 0 : s.y + 1;
    return s;
}

// Ising, bit-packed rows: bit (y, x) in word y * wpr + x / 32.
__device__ __forceinline__ uint32_t ising_bit(const uint32_t *lat, int wpr, int y, int x)
{
    return (lat[y * wpr + (x >> 5)] >> (x & 31)) & 1u;
}

// Bin change of flipping site s: dE = 2 s_i sum_j s_j (E = -sum s_i s_j), in
// bins of 4: db = s_i (n_plus - 2), n_plus = neighbours with spin +1.
__device__ __forceinline__ int ising_flip_dbin(const uint32_t *lat, int wpr, const Site &s)
{
    const int self = (int)ising_bit(lat, wpr, s.y, s.x);
    const int np = (int)(ising_bit(lat, wpr, s.y, s.xl) + ising_bit(lat, wpr, s.y, s.xr) +
                         ising_bit(lat, wpr, s.yu, s.x) + ising_bit(lat, wpr, s.yd, s.x));
    return self ? (np - 2) : (2 - np);
}

__device__ __forceinline__ void ising_flip(uint32_t *lat, int wpr, const Site &s)
{
    lat[s.y * wpr + (s.x >> 5)] ^= 1u << (s.x & 31);
}

// Potts, one byte per site.  E = -sum delta(q_i, q_j) (Eq. (2)); changing site
// i from a to v changes E by (#neighbours equal to a) - (#neighbours equal to v).
__device__ __forceinline__ int potts_get(const uint32_t *lat, int i)
{
    return (int)reinterpret_cast<const uint8_t *>(lat)[i];
}

__device__ __forceinline__ void potts_set(uint32_t *lat, int i, int v)
{
    reinterpret_cast<uint8_t *>(lat)[i] = (uint8_t)v;
}

__device__ __forceinline__ int potts_dE(const uint32_t *lat, int L, const Site &s, int old_v, int new_v)
{
    const int n0 = potts_get(lat, s.y * L + s.xl), n1 = potts_get(lat, s.y * L + s.xr);
    const int n2 = potts_get(lat, s.yu * L + s.x), n3 = potts_get(lat, s.yd * L + s.x);
    const int eq_old = (n0 == old_v) + (n1 == old_v) + (n2 == old_v) + (n3 == old_v);
    const int eq_new = (n0 == new_v) + (n1 == new_v) + (n2 == new_v) + (n3 == new_v);
    return eq_old - eq_new;
}

}  // namespace rewl
