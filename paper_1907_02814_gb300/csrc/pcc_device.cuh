// Device building blocks shared by the kernels: physical constants,
// Philox4x32-10, uniforms, the pairing permutation, status bits and warp
// helpers.  Written for sm_103a; no host fallback.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pcc.h"

namespace pcc {

// CODATA 2018.
constexpr double kAlpha = 7.2973525693e-3;       // fine-structure constant
constexpr double kRe = 2.8179403262e-15;         // classical electron radius [m]
constexpr double kRc = 3.8615926796e-13;         // reduced Compton wavelength hbar/(m_e c) [m]
constexpr double kC = 299792458.0;               // speed of light [m/s]
constexpr double kEps0 = 8.8541878128e-12;       // vacuum permittivity [F/m]
constexpr double kQe = 1.602176634e-19;          // elementary charge [C]
constexpr double kPi = 3.14159265358979323846;

// Random-stream tags: group | purpose << 4 | pass << 8 (Philox counter word 3).
enum Group : uint32_t { kGroupEm = 0, kGroupEp = 1, kGroupPh = 2 };
enum Purpose : uint32_t { kPerm = 0, kAccept = 1, kEvtBrems = 2, kEvtTri1 = 3, kEvtTri2 = 4, kEvtBH = 5,
                          kAcceptExt = 6 };
enum Channel : int { kChBremsEm = 0, kChBremsEp = 1, kChTriEm = 2, kChTriEp = 3, kChBH = 4 };

__host__ __device__ __forceinline__ uint32_t stream_tag(uint32_t group, uint32_t purpose, uint32_t pass)
{
    return group | (purpose << 4) | (pass << 8);
}

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): counter c, key k.
struct Philox4 { uint32_t v[4]; };

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // each 32 x 32 -> 64-bit product as one wide multiply
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0, m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
        const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Philox4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// Uniform on (0,1): (2m+1) 2^-24 from the top 23 bits; exact in float.
template <typename T>
__device__ __forceinline__ T u01(uint32_t r)
{
    return (T)((float)(r >> 9) + 0.5f) * (T)(1.0f / 8388608.0f);
}

__device__ __forceinline__ Philox4 draw(uint32_t c0, uint32_t cell, uint64_t step, uint32_t tag, uint64_t seed)
{
    return philox4x32_10(c0, cell, (uint32_t)step, tag, (uint32_t)seed, (uint32_t)(seed >> 32));
}

// Where the rest of an accept uniform comes from: words 0 and 1 of the draw
// (c0, cell, step, group | kAcceptExt << 4 | pass << 8) of the step's seed.
struct AcceptSrc {
    uint32_t c0, cell, tag;
};

// The accept decision U < p (Eq. proba3: collision with probability
// p = 1 - exp(-x)) for the uniform U = (2^48 a + e + 1/2) 2^-64, read digit
// by digit: the 16-bit accept digit a settles it unless a = floor(2^16 p),
// and only then (probability 2^-16) is the 48-bit rest e = 2^16 w0 +
// (w1 >> 16) drawn.  Every p is honoured down to 2^-64; a fixed-point uniform
// would drop probabilities below its resolution.  2^16 p and its fractional
// part are exact in either precision.
// The tie (a = floor(2^16 p)): the rest against frac(2^16 p) 2^48.
static __device__ __noinline__ bool accept_tie(double frac48, uint32_t c0, uint32_t cell, uint32_t tag, uint64_t step,
                                               uint64_t seed)
{
    const Philox4 e = draw(c0, cell, step, tag, seed);
    const uint64_t rest = ((uint64_t)e.v[0] << 16) | (e.v[1] >> 16);
    return (double)rest + 0.5 < frac48;
}

template <typename Real>
__device__ __forceinline__ bool accept_u(uint32_t a, Real p, const AcceptSrc& src, uint64_t step, uint64_t seed)
{
    if (!(p > (Real)0)) return false;
    if (p >= (Real)1) return true;
    const Real X = p * (Real)65536.0, fl = floor(X);
    const uint32_t u = (uint32_t)fl;
    if (a != u) return a < u;
    return accept_tie(ldexp((double)(X - fl), 48), src.c0, src.cell, src.tag, step, seed);
}

// Digit d (0..7) of an accept draw: the high (d even) or low (d odd) half of
// word d >> 1.
__device__ __forceinline__ uint32_t accept_digit(const Philox4& r, uint32_t d)
{
    const uint32_t w = r.v[(d >> 1) & 3u];
    return (d & 1u) ? (w & 0xFFFFu) : (w >> 16);
}

// Quick-reject threshold on the accept digit for a bound b >= p: a pair can
// only be accepted if a <= floor(2^16 b).  A non-finite bound lets every pair
// through to the exact evaluation.
__device__ __forceinline__ uint32_t accept_threshold(float b)
{
    const float X = b * 65536.0f;
    if (!(X < 65535.0f)) return 0xFFFFu;
    return X > 0.f ? (uint32_t)X : 0u;
}

// The same generator with the ten round keys precomputed (key schedule of
// Philox4x32-10: k0 + r 0x9E3779B9, k1 + r 0xBB67AE85), so that a kernel can
// read them from its parameter space instead of keeping them in registers.
struct PhiloxKeys { uint32_t k0[10], k1[10]; };

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ Philox4 draw_k(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, const PhiloxKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t m0 = (uint64_t)0xD2511F53u * c0, m1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)m0, hi0 = (uint32_t)(m0 >> 32);
        const uint32_t lo1 = (uint32_t)m1, hi1 = (uint32_t)(m1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ K.k0[r], n2 = hi0 ^ c3 ^ K.k1[r];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    Philox4 o;
    o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
    return o;
}

// ---------------------------------------------------------------------------
// Pairing permutation P on [0, n) for the larger list of a cell.
//   n <= 32: P^-1(s) = rank of s under keys mix(mix(s, k0), k1) (ties by s).
//   n  > 32: four-round Feistel on b = bitlen(n-1) bits with halves
//            floor(b/2), ceil(b/2) swapping widths each round, restricted to
//            [0, n) by cycle walking; P^-1 = encryption, P = decryption.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t r, uint32_t k)
{
    uint32_t t = r ^ k;
    t *= 0x9E3779B1u;
    t ^= t >> 15;
    t *= 0x85EBCA77u;
    t ^= t >> 13;
    return t;
}

struct PermKeys { uint32_t k[4]; };

__device__ __forceinline__ uint32_t small_key(uint32_t s, const PermKeys& rk)
{
    return mix32(mix32(s, rk.k[0]), rk.k[1]);
}

__device__ __forceinline__ uint32_t feistel_forward(uint32_t v, int b, const PermKeys& rk)
{
    int wl = b >> 1, wr = b - wl;
    uint32_t L = v >> wr, R = v & ((1u << wr) - 1u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const uint32_t nR = (L ^ mix32(R, rk.k[i])) & ((1u << wl) - 1u);
        L = R;
        R = nR;
        const int t = wl; wl = wr; wr = t;
    }
    return (L << wr) | R;
}

__device__ __forceinline__ uint32_t feistel_backward(uint32_t v, int b, const PermKeys& rk)
{
    int wl = b >> 1, wr = b - wl;
    uint32_t L = v >> wr, R = v & ((1u << wr) - 1u);
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        const uint32_t oL = (R ^ mix32(L, rk.k[i])) & ((1u << wr) - 1u);
        R = L;
        L = oL;
        const int t = wl; wl = wr; wr = t;
    }
    return (L << wr) | R;
}

__device__ __forceinline__ int bit_length(uint32_t v) { return v ? 32 - __clz(v) : 0; }

// P^-1(s) for n > 32 (cycle walking ends within 2^b steps: the cycle through
// s returns to s itself).
__device__ __forceinline__ uint32_t perm_pos_large(uint32_t s, uint32_t n, const PermKeys& rk)
{
    const int b = bit_length(n - 1);
    uint32_t y = feistel_forward(s, b, rk);
    for (uint32_t it = 0; y >= n && it < (1u << b); ++it) y = feistel_forward(y, b, rk);
    return y;
}

// P(j) for n > 32.
__device__ __forceinline__ uint32_t perm_elem_large(uint32_t j, uint32_t n, const PermKeys& rk)
{
    const int b = bit_length(n - 1);
    uint32_t y = feistel_backward(j, b, rk);
    for (uint32_t it = 0; y >= n && it < (1u << b); ++it) y = feistel_backward(y, b, rk);
    return y;
}

// P^-1(s) for n <= 32 by counting smaller keys.
__device__ __forceinline__ uint32_t perm_pos_small(uint32_t s, uint32_t n, const PermKeys& rk)
{
    const uint32_t ks = small_key(s, rk);
    uint32_t rank = 0;
    for (uint32_t t = 0; t < n; ++t) {
        const uint32_t kt = small_key(t, rk);
        rank += (kt < ks || (kt == ks && t < s)) ? 1u : 0u;
    }
    return rank;
}

// Secondary identifiers: marker bit | step (19 bits) | channel (3) | cell (24) | pair (16) | slot (1).
__device__ __forceinline__ uint64_t secondary_pid(uint64_t step, int ch, uint32_t cell, uint32_t j, int sub)
{
    return (1ull << 63) | ((step & 0x7FFFFull) << 44) | ((uint64_t)ch << 41) |
           ((uint64_t)(cell & 0xFFFFFFu) << 17) | ((uint64_t)(j & 0xFFFFu) << 1) | (uint64_t)sub;
}

// Device-side status and counters, one per context.
struct DevStats {
    unsigned int status;
    unsigned int pad;
    unsigned long long pairs[3];
    unsigned long long accepted[5];
    unsigned long long created[5];
    double energy_change;
    double charge_change;
    unsigned long long candidates[3];
};

__device__ __forceinline__ void raise_status(DevStats* st, unsigned bits) { atomicOr(&st->status, bits); }

// Warp reductions (fixed butterfly order: identical result on every run).
template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Kahan-compensated float accumulator.
struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

}  // namespace pcc
