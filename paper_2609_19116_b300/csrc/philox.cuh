// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and the draws of the library's
// random-number contract, usable from host and device code.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define QC_HD __host__ __device__ __forceinline__
#else
#define QC_HD inline
#endif

namespace qc {

enum : uint32_t { TAG_WORD = 0, TAG_SKIP = 1, TAG_PAULI = 2, TAG_MEAS = 3, TAG_EXACT = 4, TAG_EXACT_PAULI = 5 };

struct U4 { uint32_t x, y, z, w; };

QC_HD void mulhilo32(uint32_t a, uint32_t b, uint32_t& hi, uint32_t& lo) {
#if defined(__CUDA_ARCH__)
    hi = __umulhi(a, b);
    lo = a * b;
#else
    const uint64_t p = (uint64_t)a * (uint64_t)b;
    hi = (uint32_t)(p >> 32);
    lo = (uint32_t)p;
#endif
}

QC_HD U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(M0, c0, hi0, lo0);
        mulhilo32(M1, c2, hi1, lo1);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += W0;
        k1 += W1;
    }
    return U4{c0, c1, c2, c3};
}

QC_HD uint32_t u4_get(const U4& v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; }

// Smallest s in [0, 64) with u < tg[s], or 64.  tg is non-decreasing.
QC_HD int first_below(uint32_t u, const uint32_t* tg) {
    if (u >= tg[63]) return 64;
    int lo = 0, hi = 63;  // answer in [lo, hi]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < tg[mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Faulted lanes of channel c in word w as a 64-bit mask.  u0 is the channel's TAG_WORD draw.
QC_HD uint64_t lane_mask(uint32_t u0, uint32_t c, uint32_t w, const uint32_t* tg, uint32_t k0, uint32_t k1) {
    int lane = first_below(u0, tg);
    if (lane >= 64) return 0;
    uint64_t m = 1ull << lane;
    U4 d{0, 0, 0, 0};
    for (uint32_t k = 0;; ++k) {
        if ((k & 3) == 0) d = philox(c, w, k >> 2, TAG_SKIP, k0, k1);
        const int s = first_below(u4_get(d, k & 3), tg);
        if (s >= 64) break;
        lane += 1 + s;
        if (lane >= 64) break;
        m |= 1ull << lane;
    }
    return m;
}

// Pauli code of a faulted lane: kind 1 = DEP1 (codes 1..3), 2 = DEP2 (1..15), 3 = XERR (X).
QC_HD uint32_t fault_code(uint32_t kind, uint32_t c, uint32_t w, uint32_t lane, uint32_t k0, uint32_t k1) {
    if (kind == 3) return 1;
    const uint32_t z = (kind == 2) ? 15u : 3u;
    const uint32_t x = philox(c, w, lane, TAG_PAULI, k0, k1).x;
    return 1u + (uint32_t)(((uint64_t)x * z) >> 32);
}

// 53-bit uniform in [0, 1) for readout k of a shot.
QC_HD double readout_uniform(uint32_t k, uint64_t shot, uint32_t k0, uint32_t k1) {
    const U4 x = philox(k, (uint32_t)shot, (uint32_t)(shot >> 32), TAG_MEAS, k0, k1);
    const uint64_t u53 = ((uint64_t)(x.x >> 5) << 26) + (uint64_t)(x.y >> 6);
    return (double)u53 * (1.0 / 9007199254740992.0);
}

// Integer in [0, bound) for the fixed-weight stream (Lemire's multiply-shift with rejection);
// `draw` is the running draw counter of the shot.
QC_HD uint32_t exact_bounded(uint64_t shot, uint32_t& draw, uint32_t bound, uint32_t k0, uint32_t k1) {
    const uint32_t thresh = (uint32_t)((4294967296ull - bound) % bound);
    for (;;) {
        const uint32_t x = philox(draw, (uint32_t)shot, (uint32_t)(shot >> 32), TAG_EXACT, k0, k1).x;
        ++draw;
        const uint64_t m = (uint64_t)x * bound;
        if ((uint32_t)m >= thresh) return (uint32_t)(m >> 32);
    }
}

QC_HD uint32_t exact_code(uint32_t kind, uint32_t c, uint64_t shot, uint32_t k0, uint32_t k1) {
    if (kind == 3) return 1;
    const uint32_t z = (kind == 2) ? 15u : 3u;
    const uint32_t x = philox(c, (uint32_t)shot, (uint32_t)(shot >> 32), TAG_EXACT_PAULI, k0, k1).x;
    return 1u + (uint32_t)(((uint64_t)x * z) >> 32);
}

}  // namespace qc
