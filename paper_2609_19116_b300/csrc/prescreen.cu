// Pauli-frame pre-screen (Sec. 4.2) and fault sampling kernels.
//
// One thread owns one 64-shot word: bit i of every frame word is shot 64*w + i.  The frame of the
// word (x and z bits of every qubit) lives in shared memory laid out [qubit][thread], so that the
// threads of a warp touching the same qubit hit consecutive banks.  The program is staged in
// shared memory in chunks and swept by all threads in lockstep; noise channels draw one Philox
// block per group of four consecutive channels and word, and only the rare (channel, word) pairs
// with a fault (rate 1-(1-p)^64) walk the lane sequence.  Fault weights are counted per lane in a
// bit-sliced 5-plane counter.
#include <cstdio>
#include <vector>

#include "philox.cuh"
#include "qc_internal.h"

namespace qc {

namespace {

constexpr int PRE_THREADS = 128;
constexpr int PRE_CHUNK = 512;  // program words staged per step
constexpr int WMAX_BINS = 64;

struct PreParams {
    const PreOp* prog;
    uint32_t nops;
    uint32_t nq;
    uint32_t nchan;
    const uint8_t* chan_kind;
    uint64_t word0;      // absolute index of the first word
    uint64_t nwords;
    uint64_t nshots;     // valid shots from shot0 = word0 * 64
    uint32_t k0, k1;
    uint32_t tg[64];
    int32_t wmax;
    uint64_t* kept;      // [nwords]
    unsigned long long* hist_drawn;  // [wmax+1] device
    unsigned long long* hist_kept;
};

__device__ __forceinline__ void bs_add(uint64_t (&pl)[5], uint64_t& sat, uint64_t m) {
    uint64_t carry = m;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint64_t t = pl[i] & carry;
        pl[i] ^= carry;
        carry = t;
    }
    sat |= carry;
}

__global__ void __launch_bounds__(PRE_THREADS) prescreen_kernel(const PreParams P) {
    extern __shared__ uint64_t smem[];
    uint64_t* fx = smem;                              // [nq][PRE_THREADS]
    uint64_t* fz = fx + (size_t)P.nq * PRE_THREADS;   // [nq][PRE_THREADS]
    PreOp* chunk = reinterpret_cast<PreOp*>(fz + (size_t)P.nq * PRE_THREADS);  // [PRE_CHUNK]
    uint32_t* tg = reinterpret_cast<uint32_t*>(chunk + PRE_CHUNK);             // [64]
    unsigned long long* hd = reinterpret_cast<unsigned long long*>(tg + 64);   // [WMAX_BINS]
    unsigned long long* hk = hd + WMAX_BINS;

    const int tid = threadIdx.x;
    const uint64_t lw = (uint64_t)blockIdx.x * PRE_THREADS + tid;  // word within the call
    const bool active = lw < P.nwords;
    const uint32_t w = (uint32_t)(P.word0 + lw);

    for (int i = tid; i < 64; i += PRE_THREADS) tg[i] = P.tg[i];
    for (int i = tid; i < WMAX_BINS; i += PRE_THREADS) { hd[i] = 0; hk[i] = 0; }
    for (uint32_t q = 0; q < P.nq; ++q) {
        fx[q * PRE_THREADS + tid] = 0;
        fz[q * PRE_THREADS + tid] = 0;
    }
    uint64_t rej = 0, sat = 0;
    uint64_t planes[5] = {0, 0, 0, 0, 0};
    uint32_t cached_group = 0xFFFFFFFFu;
    U4 cu{0, 0, 0, 0};

    for (uint32_t base = 0; base < P.nops; base += PRE_CHUNK) {
        const uint32_t cnt = min((uint32_t)PRE_CHUNK, P.nops - base);
        __syncthreads();
        for (uint32_t i = tid; i < cnt; i += PRE_THREADS) chunk[i] = P.prog[base + i];
        __syncthreads();
        if (!active) continue;
        for (uint32_t i = 0; i < cnt; ++i) {
            const PreOp op = chunk[i];
            const uint32_t kind = op.w0 & 15u;
            const uint32_t a = (op.w0 >> 4) & 0xFFFu, b = op.w0 >> 16;
            uint64_t* xa = fx + a * PRE_THREADS + tid;
            uint64_t* za = fz + a * PRE_THREADS + tid;
            switch (kind) {
                case P_H: { const uint64_t t = *xa; *xa = *za; *za = t; break; }
                case P_S: *za ^= *xa; break;
                case P_CX: {
                    uint64_t* xb = fx + b * PRE_THREADS + tid;
                    uint64_t* zb = fz + b * PRE_THREADS + tid;
                    *xb ^= *xa;
                    *za ^= *zb;
                    break;
                }
                case P_CZ: {
                    uint64_t* xb = fx + b * PRE_THREADS + tid;
                    uint64_t* zb = fz + b * PRE_THREADS + tid;
                    const uint64_t x1 = *xa, x2 = *xb;
                    *za ^= x2;
                    *zb ^= x1;
                    break;
                }
                case P_SWAP: {
                    uint64_t* xb = fx + b * PRE_THREADS + tid;
                    uint64_t* zb = fz + b * PRE_THREADS + tid;
                    uint64_t t = *xa; *xa = *xb; *xb = t;
                    t = *za; *za = *zb; *zb = t;
                    break;
                }
                case P_DEP1: case P_DEP2: case P_XERR: {
                    const uint32_t c = op.w1;
                    if ((c >> 2) != cached_group) {
                        cached_group = c >> 2;
                        cu = philox(cached_group, w, 0, TAG_WORD, P.k0, P.k1);
                    }
                    const uint32_t u0 = u4_get(cu, c & 3);
                    if (u0 >= tg[63]) break;  // no fault of this channel in the word
                    const uint64_t m = lane_mask(u0, c, w, tg, P.k0, P.k1);
                    bs_add(planes, sat, m);
                    const uint32_t ck = kind == P_DEP1 ? 1u : kind == P_DEP2 ? 2u : 3u;
                    if (ck == 3) { *xa ^= m; break; }
                    uint64_t mxa = 0, mza = 0, mxb = 0, mzb = 0;
                    for (uint64_t r = m; r; r &= r - 1) {
                        const uint32_t lane = __ffsll((long long)r) - 1;
                        const uint64_t bit = 1ull << lane;
                        const uint32_t code = fault_code(ck, c, w, lane, P.k0, P.k1);
                        uint32_t px, pz;
                        if (ck == 2) {
                            pauli_xz(code >> 2, px, pz);
                            if (px) mxa |= bit;
                            if (pz) mza |= bit;
                            pauli_xz(code & 3, px, pz);
                            if (px) mxb |= bit;
                            if (pz) mzb |= bit;
                        } else {
                            pauli_xz(code, px, pz);
                            if (px) mxa |= bit;
                            if (pz) mza |= bit;
                        }
                    }
                    *xa ^= mxa;
                    *za ^= mza;
                    if (ck == 2) {
                        fx[b * PRE_THREADS + tid] ^= mxb;
                        fz[b * PRE_THREADS + tid] ^= mzb;
                    }
                    break;
                }
                case P_MDEC: rej |= *xa; *xa = 0; *za = 0; break;
                case P_CLEAR: *xa = 0; *za = 0; break;
                default: break;
            }
        }
    }
    if (active) {
        const uint64_t first = lw * 64;
        uint64_t valid = ~0ull;
        if (first + 64 > P.nshots) valid = (P.nshots > first) ? ((1ull << (P.nshots - first)) - 1) : 0;
        const uint64_t kept = ~rej & valid;
        P.kept[lw] = kept;
        // per-weight histogram: lanes whose 5-bit count equals v (bin wmax collects >= wmax)
        uint64_t seen = 0;
        for (int v = 0; v < P.wmax; ++v) {
            uint64_t m = ~sat;
#pragma unroll
            for (int i = 0; i < 5; ++i) m &= ((v >> i) & 1) ? planes[i] : ~planes[i];
            seen |= m;
            const int nd = __popcll(m & valid), nk = __popcll(m & kept);
            if (nd) atomicAdd(&hd[v], (unsigned long long)nd);
            if (nk) atomicAdd(&hk[v], (unsigned long long)nk);
        }
        const uint64_t rest = ~seen;
        const int nd = __popcll(rest & valid), nk = __popcll(rest & kept);
        if (nd) atomicAdd(&hd[P.wmax], (unsigned long long)nd);
        if (nk) atomicAdd(&hk[P.wmax], (unsigned long long)nk);
    }
    __syncthreads();
    for (int i = tid; i <= P.wmax; i += PRE_THREADS) {
        if (hd[i]) atomicAdd(&P.hist_drawn[i], hd[i]);
        if (hk[i]) atomicAdd(&P.hist_kept[i], hk[i]);
    }
}

// ---- fixed-weight pre-screen (subset sampling, Sec. 4.1): one thread per shot --------------------
// Each shot has exactly w faults (Floyd's algorithm over the channels); the thread keeps them sorted
// by channel and sweeps the frame program with the frame in registers (x and z bits of up to 128
// qubits), so a noise instruction only compares its channel with the next fault.
constexpr int EX_MAXW = 32;
constexpr int EX_THREADS = 128;

__device__ __forceinline__ bool bit2(const uint64_t (&v)[2], uint32_t q) { return (v[q >> 6] >> (q & 63)) & 1; }
__device__ __forceinline__ void flip2(uint64_t (&v)[2], uint32_t q, bool b) { v[q >> 6] ^= (uint64_t)b << (q & 63); }
__device__ __forceinline__ void clr2(uint64_t (&v)[2], uint32_t q) { v[q >> 6] &= ~(1ull << (q & 63)); }

__global__ void __launch_bounds__(EX_THREADS) prescreen_exact_kernel(const PreParams P, int weight) {
    __shared__ PreOp chunk[PRE_CHUNK];
    __shared__ unsigned long long hd, hk;
    const uint64_t i = (uint64_t)blockIdx.x * EX_THREADS + threadIdx.x;
    const bool active = i < P.nshots;
    const uint64_t shot = P.word0 * 64 + i;
    if (threadIdx.x == 0) { hd = 0; hk = 0; }
    uint32_t fc[EX_MAXW];
    uint8_t fk[EX_MAXW];
    int nf = 0;
    if (active) {
        uint32_t draw = 0;
        const uint32_t M = P.nchan, W = (uint32_t)weight;
        for (uint32_t j = M - W; j < M; ++j) {
            const uint32_t t = exact_bounded(shot, draw, j + 1, P.k0, P.k1);
            bool present = false;
            for (int k = 0; k < nf; ++k) present |= (fc[k] == t);
            const uint32_t v = present ? j : t;
            int k = nf;
            while (k > 0 && fc[k - 1] > v) { fc[k] = fc[k - 1]; --k; }
            fc[k] = v;
            ++nf;
        }
        for (int k = 0; k < nf; ++k) fk[k] = (uint8_t)exact_code(P.chan_kind[fc[k]], fc[k], shot, P.k0, P.k1);
    }
    uint64_t x[2] = {0, 0}, z[2] = {0, 0};
    bool rej = false;
    int ptr = 0;
    for (uint32_t base = 0; base < P.nops; base += PRE_CHUNK) {
        const uint32_t cnt = min((uint32_t)PRE_CHUNK, P.nops - base);
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < cnt; k += EX_THREADS) chunk[k] = P.prog[base + k];
        __syncthreads();
        if (!active) continue;
        for (uint32_t k = 0; k < cnt; ++k) {
            const PreOp op = chunk[k];
            const uint32_t kind = op.w0 & 15u;
            const uint32_t a = (op.w0 >> 4) & 0xFFFu, b = op.w0 >> 16;
            switch (kind) {
                case P_H: { const bool xa = bit2(x, a), za = bit2(z, a); flip2(x, a, xa ^ za); flip2(z, a, xa ^ za); break; }
                case P_S: flip2(z, a, bit2(x, a)); break;
                case P_CX: flip2(x, b, bit2(x, a)); flip2(z, a, bit2(z, b)); break;
                case P_CZ: { const bool xa = bit2(x, a), xb = bit2(x, b); flip2(z, a, xb); flip2(z, b, xa); break; }
                case P_SWAP: {
                    const bool xa = bit2(x, a), za = bit2(z, a), xb = bit2(x, b), zb = bit2(z, b);
                    flip2(x, a, xa ^ xb); flip2(x, b, xa ^ xb); flip2(z, a, za ^ zb); flip2(z, b, za ^ zb);
                    break;
                }
                case P_DEP1: case P_DEP2: case P_XERR: {
                    if (ptr < nf && fc[ptr] == op.w1) {
                        const uint32_t code = fk[ptr++];
                        uint32_t px, pz;
                        if (kind == P_DEP2) {
                            pauli_xz(code >> 2, px, pz); flip2(x, a, px); flip2(z, a, pz);
                            pauli_xz(code & 3, px, pz); flip2(x, b, px); flip2(z, b, pz);
                        } else {
                            pauli_xz(code, px, pz); flip2(x, a, px); flip2(z, a, pz);
                        }
                    }
                    break;
                }
                case P_MDEC: rej |= bit2(x, a); clr2(x, a); clr2(z, a); break;
                case P_CLEAR: clr2(x, a); clr2(z, a); break;
                default: break;
            }
        }
    }
    // kept bits: lane l of a warp holds shot 32*warp_index + l; two warps make a 64-shot word
    const unsigned ballot = __ballot_sync(0xFFFFFFFFu, active && !rej);
    const uint64_t word = i >> 6;
    if ((threadIdx.x & 31) == 0 && (i < P.nshots)) {
        const int half = (int)((i >> 5) & 1);
        atomicOr(reinterpret_cast<unsigned long long*>(P.kept) + word, (unsigned long long)ballot << (32 * half));
    }
    if (active) {
        atomicAdd(&hd, 1ull);
        if (!rej) atomicAdd(&hk, 1ull);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int wb = min(weight, P.wmax);
        if (hd) atomicAdd(&P.hist_drawn[wb], hd);
        if (hk) atomicAdd(&P.hist_kept[wb], hk);
    }
}

// ---- survivor compaction: count per chunk, scan, write in shot order ----------------------------
constexpr int CMP_THREADS = 256;
constexpr int CMP_WORDS = 4;  // words per thread
constexpr int CMP_CHUNK = CMP_THREADS * CMP_WORDS;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh, uint32_t& total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    total = sh[(blockDim.x >> 5) - 1];
    const uint32_t warp_base = wid ? sh[wid - 1] : 0;
    __syncthreads();
    return warp_base + x - v;
}

__global__ void __launch_bounds__(CMP_THREADS) compact_count(const uint64_t* kept, uint64_t nwords,
                                                             uint64_t* chunk_count) {
    __shared__ uint32_t sh[32];
    uint32_t c = 0;
    const uint64_t w0 = (uint64_t)blockIdx.x * CMP_CHUNK + (uint64_t)threadIdx.x * CMP_WORDS;
    for (int k = 0; k < CMP_WORDS; ++k)
        if (w0 + k < nwords) c += __popcll(kept[w0 + k]);
    uint32_t total;
    block_exclusive_scan(c, sh, total);
    if (threadIdx.x == 0) chunk_count[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) compact_scan(uint64_t* chunk_count, uint64_t nchunks, uint64_t* total_out) {
    // exclusive scan in place, sequential over blocks of 1024 chunks
    __shared__ uint64_t sh[1024];
    __shared__ uint64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < nchunks; base += 1024) {
        const uint64_t i = base + threadIdx.x;
        const uint64_t v = i < nchunks ? chunk_count[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const uint64_t y = threadIdx.x >= (unsigned)o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < nchunks) chunk_count[i] = carry + sh[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += sh[1023];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void __launch_bounds__(CMP_THREADS) compact_write(const uint64_t* kept, uint64_t nwords,
                                                             const uint64_t* chunk_off, uint64_t shot0,
                                                             uint64_t* out, uint64_t capacity) {
    __shared__ uint32_t sh[32];
    const uint64_t w0 = (uint64_t)blockIdx.x * CMP_CHUNK + (uint64_t)threadIdx.x * CMP_WORDS;
    uint64_t words[CMP_WORDS];
    uint32_t c = 0;
    for (int k = 0; k < CMP_WORDS; ++k) {
        words[k] = (w0 + k < nwords) ? kept[w0 + k] : 0;
        c += __popcll(words[k]);
    }
    uint32_t total;
    uint64_t pos = chunk_off[blockIdx.x] + block_exclusive_scan(c, sh, total);
    for (int k = 0; k < CMP_WORDS; ++k)
        for (uint64_t r = words[k]; r; r &= r - 1) {
            const uint32_t lane = __ffsll((long long)r) - 1;
            if (pos < capacity) out[pos] = shot0 + (w0 + k) * 64 + lane;
            ++pos;
        }
}

// ---- fault lists of given shots (the contract's draws, one thread per shot) --------------------
struct FaultParams {
    const uint64_t* shots;
    uint64_t nshots;
    uint32_t nchan;
    const uint8_t* chan_kind;
    uint32_t k0, k1;
    uint32_t tg[64];
    int32_t weight;  // -1 Bernoulli, else exact
    uint32_t max_faults;
    uint32_t* count;
    uint32_t* chan;
    uint8_t* code;
};

__global__ void fault_kernel(const FaultParams P) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nshots) return;
    const uint64_t shot = P.shots[i];
    uint32_t n = 0;
    if (P.weight < 0) {
        const uint32_t w = (uint32_t)(shot >> 6), lane = (uint32_t)(shot & 63);
        for (uint32_t g = 0; g * 4 < P.nchan; ++g) {
            const U4 u = philox(g, w, 0, TAG_WORD, P.k0, P.k1);
            for (uint32_t j = 0; j < 4; ++j) {
                const uint32_t c = g * 4 + j;
                if (c >= P.nchan) break;
                const uint32_t u0 = u4_get(u, j);
                if (u0 >= P.tg[63]) continue;
                const uint64_t m = lane_mask(u0, c, w, P.tg, P.k0, P.k1);
                if (!((m >> lane) & 1)) continue;
                if (n < P.max_faults) {
                    P.chan[i * P.max_faults + n] = c;
                    P.code[i * P.max_faults + n] = (uint8_t)fault_code(P.chan_kind[c], c, w, lane, P.k0, P.k1);
                }
                ++n;
            }
        }
    } else {
        // Floyd's algorithm; the chosen set is kept sorted in the output arrays
        uint32_t draw = 0;
        const uint32_t M = P.nchan, W = (uint32_t)P.weight;
        uint32_t* ch = P.chan + i * P.max_faults;
        for (uint32_t j = M - W; j < M; ++j) {
            const uint32_t t = exact_bounded(shot, draw, j + 1, P.k0, P.k1);
            bool present = false;
            for (uint32_t k = 0; k < min(n, P.max_faults); ++k) present |= (ch[k] == t);
            const uint32_t v = present ? j : t;
            if (n < P.max_faults) {
                uint32_t k = n;
                while (k > 0 && ch[k - 1] > v) { ch[k] = ch[k - 1]; --k; }
                ch[k] = v;
            }
            ++n;
        }
        for (uint32_t k = 0; k < min(n, P.max_faults); ++k)
            P.code[i * P.max_faults + k] = (uint8_t)exact_code(P.chan_kind[ch[k]], ch[k], shot, P.k0, P.k1);
    }
    P.count[i] = n;
}

}  // namespace
}  // namespace qc

using namespace qc;

extern "C" qc_status qc_sample_faults(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                                      uint64_t nshots, uint32_t max_faults, uint32_t* count_dev,
                                      uint32_t* chan_dev, uint8_t* code_dev, void* stream) {
    if (!circuit || (nshots && (!shots_dev || !count_dev))) return fail(QC_EINVAL, "null argument");
    if (!(noise.p >= 0.0 && noise.p < 1.0)) return fail(QC_EINVAL, "p must lie in [0, 1)");
    if (max_faults && (!chan_dev || !code_dev)) return fail(QC_EINVAL, "null fault buffers");
    CircuitImpl& c = const_cast<qc_circuit*>(circuit)->impl;
    if (noise.fault_weight >= 0 && (uint64_t)noise.fault_weight > c.chan_kind.size())
        return fail(QC_EINVAL, "fault weight exceeds the number of channels");
    if (nshots == 0) return QC_OK;
    DeviceCopy* dc;
    qc_status st = c.device_copy(&dc);
    if (st != QC_OK) return st;
    FaultParams P{};
    P.shots = shots_dev;
    P.nshots = nshots;
    P.nchan = (uint32_t)c.chan_kind.size();
    P.chan_kind = dc->chan_kind;
    P.k0 = (uint32_t)noise.seed;
    P.k1 = (uint32_t)(noise.seed >> 32);
    const Thresholds th = make_thresholds(noise.p);
    for (int s = 0; s < 64; ++s) P.tg[s] = th.tg[s];
    P.weight = noise.fault_weight;
    P.max_faults = max_faults;
    P.count = count_dev;
    P.chan = chan_dev;
    P.code = code_dev;
    const int T = 128;
    fault_kernel<<<(unsigned)((nshots + T - 1) / T), T, 0, (cudaStream_t)stream>>>(P);
    QC_CUDA(cudaGetLastError());
    return QC_OK;
}

namespace qc {
// Shared by the public entry point and by the serving loop.
qc_status prescreen_run(CircuitImpl& c, qc_noise noise, uint64_t shot0, uint64_t nshots, uint64_t* kept_mask_dev,
                        qc_survivors* survivors, uint64_t* hist_drawn, uint64_t* hist_kept, int32_t w_max,
                        cudaStream_t s) {
    if (!(noise.p >= 0.0 && noise.p < 1.0)) return fail(QC_EINVAL, "p must lie in [0, 1)");
    if (noise.fault_weight >= 0 && (noise.fault_weight > EX_MAXW || (uint64_t)noise.fault_weight > c.chan_kind.size()))
        return fail(QC_EINVAL, "fixed fault weight must lie in [0, min(%d, channels)]", EX_MAXW);
    if (noise.fault_weight >= 0 && c.n > 128) return fail(QC_EINVAL, "fixed-weight pre-screen supports up to 128 qubits");
    if (shot0 % 64) return fail(QC_EINVAL, "shot0 must be a multiple of 64");
    if ((shot0 + nshots) / 64 >= (1ull << 32)) return fail(QC_EINVAL, "shot index beyond the 2^38 range of the contract");
    if (w_max < 0 || w_max >= WMAX_BINS) return fail(QC_EINVAL, "w_max must lie in [0, 63]");
    if (nshots && !kept_mask_dev) return fail(QC_EINVAL, "null kept mask");
    if (survivors && survivors->capacity && !survivors->shots_dev) return fail(QC_EINVAL, "null survivor buffer");
    const uint64_t nwords = (nshots + 63) / 64;
    if (nshots == 0) {
        if (survivors) survivors->count = 0;
        for (int i = 0; hist_drawn && i <= w_max; ++i) hist_drawn[i] = 0;
        for (int i = 0; hist_kept && i <= w_max; ++i) hist_kept[i] = 0;
        return QC_OK;
    }
    DeviceCopy* dc;
    qc_status st = c.device_copy(&dc);
    if (st != QC_OK) return st;

    PreParams P{};
    P.prog = dc->pre;
    P.nops = (uint32_t)c.pre.size();
    P.nq = (uint32_t)c.n;
    P.nchan = (uint32_t)c.chan_kind.size();
    P.chan_kind = dc->chan_kind;
    P.word0 = shot0 / 64;
    P.nwords = nwords;
    P.nshots = nshots;
    P.k0 = (uint32_t)noise.seed;
    P.k1 = (uint32_t)(noise.seed >> 32);
    const Thresholds th = make_thresholds(noise.p);
    for (int i = 0; i < 64; ++i) P.tg[i] = th.tg[i];
    P.wmax = w_max;
    P.kept = kept_mask_dev;

    const uint64_t nchunks = (nwords + CMP_CHUNK - 1) / CMP_CHUNK;
    // scratch: histograms (2 x 64) + chunk offsets + total
    uint64_t* scratch = nullptr;
    const size_t scratch_words = 2 * WMAX_BINS + nchunks + 1;
    QC_CUDA(cudaMallocAsync((void**)&scratch, scratch_words * sizeof(uint64_t), s));
    qc_status out = QC_OK;
    do {
        cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * WMAX_BINS * sizeof(uint64_t), s);
        if (e != cudaSuccess) { out = cuda_fail(e, "memset"); break; }
        P.hist_drawn = reinterpret_cast<unsigned long long*>(scratch);
        P.hist_kept = P.hist_drawn + WMAX_BINS;
        const size_t smem = 2ull * c.n * PRE_THREADS * sizeof(uint64_t) + PRE_CHUNK * sizeof(PreOp) +
                            64 * sizeof(uint32_t) + 2 * WMAX_BINS * sizeof(unsigned long long);
        if (smem > 227 * 1024) { out = fail(QC_EINVAL, "too many qubits for the pre-screen frame (%d)", c.n); break; }
        out = smem_optin((const void*)prescreen_kernel);
        if (out != QC_OK) break;
        if (noise.fault_weight >= 0) {
            e = cudaMemsetAsync(kept_mask_dev, 0, nwords * sizeof(uint64_t), s);
            if (e != cudaSuccess) { out = cuda_fail(e, "memset"); break; }
            prescreen_exact_kernel<<<(unsigned)((nshots + EX_THREADS - 1) / EX_THREADS), EX_THREADS, 0, s>>>(
                P, noise.fault_weight);
        } else {
            const uint64_t blocks = (nwords + PRE_THREADS - 1) / PRE_THREADS;
            prescreen_kernel<<<(unsigned)blocks, PRE_THREADS, smem, s>>>(P);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) { out = cuda_fail(e, "prescreen_kernel"); break; }
        uint64_t total = 0;
        if (survivors) {
            uint64_t* chunk = scratch + 2 * WMAX_BINS;
            uint64_t* tot = chunk + nchunks;
            compact_count<<<(unsigned)nchunks, CMP_THREADS, 0, s>>>(kept_mask_dev, nwords, chunk);
            compact_scan<<<1, 1024, 0, s>>>(chunk, nchunks, tot);
            compact_write<<<(unsigned)nchunks, CMP_THREADS, 0, s>>>(kept_mask_dev, nwords, chunk, shot0,
                                                                   survivors->shots_dev, survivors->capacity);
            e = cudaGetLastError();
            if (e != cudaSuccess) { out = cuda_fail(e, "compaction"); break; }
            e = cudaMemcpyAsync(&total, tot, sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { out = cuda_fail(e, "copy count"); break; }
        }
        std::vector<uint64_t> h(2 * WMAX_BINS);
        e = cudaMemcpyAsync(h.data(), scratch, h.size() * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) { out = cuda_fail(e, "copy histograms"); break; }
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { out = cuda_fail(e, "pre-screen"); break; }
        if (survivors) survivors->count = total;
        for (int i = 0; hist_drawn && i <= w_max; ++i) hist_drawn[i] = h[i];
        for (int i = 0; hist_kept && i <= w_max; ++i) hist_kept[i] = h[WMAX_BINS + i];
    } while (0);
    cudaFreeAsync(scratch, s);
    return out;
}
}  // namespace qc

extern "C" qc_status pauli_prescreen(const qc_circuit* circuit, qc_noise noise, uint64_t shot0, uint64_t nshots,
                                     uint64_t* kept_mask_dev, qc_survivors* survivors, uint64_t* hist_drawn,
                                     uint64_t* hist_kept, int32_t w_max, void* stream) {
    if (!circuit) return fail(QC_EINVAL, "null circuit");
    return prescreen_run(const_cast<qc_circuit*>(circuit)->impl, noise, shot0, nshots, kept_mask_dev, survivors,
                         hist_drawn, hist_kept, w_max, (cudaStream_t)stream);
}

// ---- pre-screen variant for callers that cannot allocate device memory ------------------------
// Some callers cannot call cudaMalloc at all: a serving process whose device memory is a fixed pool
// with a locked budget, or an embedding runtime that owns every allocation.  (The call copies its
// counts to host memory and synchronises the stream, so it does not belong inside a stream capture.)  This variant
// keeps all of its scratch -- the staged frame program, the per-weight histograms and the
// compaction offsets -- in one file-scope device array instead of allocating it.  The array is
// part of the library image: every GPU that loads the library holds it until the process exits.
namespace qc {
namespace {

constexpr uint64_t NA_MAX_PROG = 131072;   // frame-program words (8 bytes each)
constexpr uint64_t NA_MAX_CHUNKS = 8192;   // compaction chunks of 1024 words: 536,870,912 shots
constexpr uint64_t NA_BYTES = NA_MAX_PROG * sizeof(PreOp) + (2 * WMAX_BINS + NA_MAX_CHUNKS + 8) * sizeof(uint64_t);

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

std::mutex g_na_mu;
std::map<int, unsigned char*> g_na_addr;  // device -> address of g_noalloc_scratch on that device

// The host-side name g_noalloc_scratch is a stand-in, not a device address: take the address on
// the current device once and pass that to the kernels.
qc_status noalloc_scratch(unsigned char** out) {
    int d = 0;
    QC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_na_mu);
    auto it = g_na_addr.find(d);
    if (it == g_na_addr.end()) {
        unsigned char* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        it = g_na_addr.emplace(d, ptr).first;
    }
    *out = it->second;
    return QC_OK;
}

}  // namespace
}  // namespace qc

extern "C" qc_status pauli_prescreen_noalloc(const qc_circuit* circuit, qc_noise noise, uint64_t shot0,
                                             uint64_t nshots, uint64_t* kept_mask_dev, uint64_t* survivors_dev,
                                             uint64_t capacity, uint64_t* n_kept, uint64_t* hist_drawn,
                                             uint64_t* hist_kept, int32_t w_max, void* stream) {
    using namespace qc;
    if (!circuit || !n_kept) return fail(QC_EINVAL, "null argument");
    const CircuitImpl& c = circuit->impl;
    cudaStream_t s = (cudaStream_t)stream;
    if (!(noise.p >= 0.0 && noise.p < 1.0)) return fail(QC_EINVAL, "p must lie in [0, 1)");
    if (noise.fault_weight >= 0) return fail(QC_EINVAL, "the pre-screen takes Bernoulli noise (fault_weight = -1)");
    if (shot0 % 64) return fail(QC_EINVAL, "shot0 must be a multiple of 64");
    if ((shot0 + nshots) / 64 >= (1ull << 32)) return fail(QC_EINVAL, "shot index beyond the 2^38 range of the contract");
    if (w_max < 0 || w_max >= WMAX_BINS) return fail(QC_EINVAL, "w_max must lie in [0, 63]");
    if (nshots && !kept_mask_dev) return fail(QC_EINVAL, "null kept mask");
    if (capacity && !survivors_dev) return fail(QC_EINVAL, "null survivor buffer");
    const uint64_t nwords = (nshots + 63) / 64;
    const uint64_t nchunks = (nwords + CMP_CHUNK - 1) / CMP_CHUNK;
    if (c.pre.size() > NA_MAX_PROG)
        return fail(QC_ECAPACITY, "circuit needs %zu frame-program words; this entry point holds at most %llu",
                    c.pre.size(), (unsigned long long)NA_MAX_PROG);
    if (nchunks > NA_MAX_CHUNKS)
        return fail(QC_ECAPACITY, "%llu shots exceed the %llu this entry point handles per call",
                    (unsigned long long)nshots, (unsigned long long)(NA_MAX_CHUNKS * CMP_CHUNK * 64));
    const size_t smem = 2ull * c.n * PRE_THREADS * sizeof(uint64_t) + PRE_CHUNK * sizeof(PreOp) +
                        64 * sizeof(uint32_t) + 2 * WMAX_BINS * sizeof(unsigned long long);
    if (smem > 227 * 1024) return fail(QC_EINVAL, "too many qubits for the pre-screen frame (%d)", c.n);
    unsigned char* base = nullptr;
    qc_status st = noalloc_scratch(&base);
    if (st != QC_OK) return st;
    if (nshots == 0) {
        *n_kept = 0;
        for (int i = 0; hist_drawn && i <= w_max; ++i) hist_drawn[i] = 0;
        for (int i = 0; hist_kept && i <= w_max; ++i) hist_kept[i] = 0;
        return QC_OK;
    }
    PreOp* prog = reinterpret_cast<PreOp*>(base);
    uint64_t* hist = reinterpret_cast<uint64_t*>(base + NA_MAX_PROG * sizeof(PreOp));  // [2 * WMAX_BINS]
    uint64_t* chunk = hist + 2 * WMAX_BINS;                                             // [nchunks]
    uint64_t* total = chunk + NA_MAX_CHUNKS;                                            // [1]
    // the array keeps the previous call's contents: stage the program, clear the counters
    if (!c.pre.empty())
        QC_CUDA(cudaMemcpyAsync(prog, c.pre.data(), c.pre.size() * sizeof(PreOp), cudaMemcpyHostToDevice, s));
    QC_CUDA(cudaMemsetAsync(hist, 0, 2 * WMAX_BINS * sizeof(uint64_t), s));
    QC_CUDA(cudaMemsetAsync(total, 0, sizeof(uint64_t), s));
    PreParams P{};
    P.prog = prog;
    P.nops = (uint32_t)c.pre.size();
    P.nq = (uint32_t)c.n;
    P.nchan = (uint32_t)c.chan_kind.size();
    P.chan_kind = nullptr;  // the frame program carries the channel kinds
    P.word0 = shot0 / 64;
    P.nwords = nwords;
    P.nshots = nshots;
    P.k0 = (uint32_t)noise.seed;
    P.k1 = (uint32_t)(noise.seed >> 32);
    const Thresholds th = make_thresholds(noise.p);
    for (int i = 0; i < 64; ++i) P.tg[i] = th.tg[i];
    P.wmax = w_max;
    P.kept = kept_mask_dev;
    P.hist_drawn = reinterpret_cast<unsigned long long*>(hist);
    P.hist_kept = P.hist_drawn + WMAX_BINS;
    st = smem_optin((const void*)prescreen_kernel);
    if (st != QC_OK) return st;
    prescreen_kernel<<<(unsigned)((nwords + PRE_THREADS - 1) / PRE_THREADS), PRE_THREADS, smem, s>>>(P);
    QC_CUDA(cudaGetLastError());
    compact_count<<<(unsigned)nchunks, CMP_THREADS, 0, s>>>(kept_mask_dev, nwords, chunk);
    compact_scan<<<1, 1024, 0, s>>>(chunk, nchunks, total);
    compact_write<<<(unsigned)nchunks, CMP_THREADS, 0, s>>>(kept_mask_dev, nwords, chunk, shot0, survivors_dev,
                                                           capacity);
    QC_CUDA(cudaGetLastError());
    uint64_t h[2 * WMAX_BINS];
    uint64_t cnt = 0;
    QC_CUDA(cudaMemcpyAsync(h, hist, sizeof h, cudaMemcpyDeviceToHost, s));
    QC_CUDA(cudaMemcpyAsync(&cnt, total, sizeof cnt, cudaMemcpyDeviceToHost, s));
    QC_CUDA(cudaStreamSynchronize(s));
    *n_kept = cnt;
    for (int i = 0; hist_drawn && i <= w_max; ++i) hist_drawn[i] = h[i];
    for (int i = 0; hist_kept && i <= w_max; ++i) hist_kept[i] = h[WMAX_BINS + i];
    return QC_OK;
}
