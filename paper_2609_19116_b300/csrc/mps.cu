// Batched MPS shot engine (Sec. 3.1, Sec. 4, Sec. 4.3).
//
// Persistent launch: every CTA owns one shot slot (its site tensors in HBM plus a split scratch)
// and pulls shot indices from a global counter until none is left, so a shot that post-selection
// rejects early frees its slot at once for the next one (online screening, Sec. 4.3).  A shot walks
// the compiled site-operation program: single-site gates in place; a two-site update contracts
// the pair into theta (2chi_l x 2chi_r), applies the 4x4 gate and splits it by a one-sided
// (Hestenes) Jacobi SVD held in shared memory whenever theta fits there; readouts take the
// Born probability of the orthogonality-centre tensor in FP64.  At the end the normalised overlap
// with the noiseless reference state decides the logical-error flag (Sec. 4, App. A.3).
//
// The split avoids accumulating V: Jacobi orthogonalises the columns of theta (centre moving
// right) or of theta^H (centre moving left); the orthonormal factor is kept, and the centre
// tensor is the projection of the saved theta on it.
#include <cfloat>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "philox.cuh"
#include "qc_internal.h"
#include "tc.cuh"

namespace qc {
namespace {

template <typename R> struct VecOf;
template <> struct VecOf<float> { using T = float2; };
template <> struct VecOf<double> { using T = double2; };

template <typename V> __device__ __forceinline__ V cmk(decltype(V::x) a, decltype(V::x) b) { V v; v.x = a; v.y = b; return v; }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) { return cmk<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) { return cmk<V>(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x); }  // conj(a)*b
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmk<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V cfma(V a, V b, V c) {  // a*b + c
    return cmk<V>(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
template <typename V> __device__ __forceinline__ V cfmac(V a, V b, V c) {  // conj(a)*b + c
    return cmk<V>(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}

// sum_i conj(u[i]) t[i * ts] and sum_i t[i * ts] u[i] over n terms, as two interleaved partial sums (even
// and odd i) so that two dependent complex-FMA chains run side by side; complex64 uses the paired FP32 FMA
// (real and imaginary parts in one 64-bit register).
template <typename V>
__device__ __forceinline__ V dot_conj(const V* u, const V* t, size_t ts, int n) {
    if constexpr (sizeof(V) == 8) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
        int i = 0;
        const V* tp = t;  // t[i * ts] walked by pointer
#pragma unroll 1
        for (; i + 1 < n; i += 2, tp += 2 * ts) {
            const float2 x0 = u[i], y0 = tp[0], x1 = u[i + 1], y1 = tp[ts];
            a0 = __ffma2_rn(make_float2(x0.x, x0.x), y0, a0);                      // (ux tx, ux ty)
            b0 = __ffma2_rn(make_float2(x0.y, -x0.y), make_float2(y0.y, y0.x), b0);  // (uy ty, -uy tx)
            a1 = __ffma2_rn(make_float2(x1.x, x1.x), y1, a1);
            b1 = __ffma2_rn(make_float2(x1.y, -x1.y), make_float2(y1.y, y1.x), b1);
        }
        if (i < n) {
            const float2 x0 = u[i], y0 = tp[0];
            a0 = __ffma2_rn(make_float2(x0.x, x0.x), y0, a0);
            b0 = __ffma2_rn(make_float2(x0.y, -x0.y), make_float2(y0.y, y0.x), b0);
        }
        const float2 s = __fadd2_rn(__fadd2_rn(a0, a1), __fadd2_rn(b0, b1));
        return cmk<V>(s.x, s.y);
    } else {
        V a0 = cmk<V>(0, 0), a1 = a0;
        int i = 0;
#pragma unroll 1
        for (; i + 1 < n; i += 2) {
            a0 = cfmac(u[i], t[(size_t)i * ts], a0);
            a1 = cfmac(u[i + 1], t[(size_t)(i + 1) * ts], a1);
        }
        if (i < n) a0 = cfmac(u[i], t[(size_t)i * ts], a0);
        return cadd(a0, a1);
    }
}
template <typename V>
__device__ __forceinline__ V dot_plain(const V* t, const V* u, int n) {  // sum_i t[i] u[i]
    if constexpr (sizeof(V) == 8) {
        float2 a0 = make_float2(0.f, 0.f), a1 = a0, b0 = a0, b1 = a0;
        int i = 0;
#pragma unroll 1
        for (; i + 1 < n; i += 2) {
            const float2 x0 = t[i], y0 = u[i], x1 = t[i + 1], y1 = u[i + 1];
            a0 = __ffma2_rn(make_float2(x0.x, x0.x), y0, a0);                       // (tx ux, tx uy)
            b0 = __ffma2_rn(make_float2(-x0.y, x0.y), make_float2(y0.y, y0.x), b0);  // (-ty uy, ty ux)
            a1 = __ffma2_rn(make_float2(x1.x, x1.x), y1, a1);
            b1 = __ffma2_rn(make_float2(-x1.y, x1.y), make_float2(y1.y, y1.x), b1);
        }
        if (i < n) {
            const float2 x0 = t[i], y0 = u[i];
            a0 = __ffma2_rn(make_float2(x0.x, x0.x), y0, a0);
            b0 = __ffma2_rn(make_float2(-x0.y, x0.y), make_float2(y0.y, y0.x), b0);
        }
        const float2 s = __fadd2_rn(__fadd2_rn(a0, a1), __fadd2_rn(b0, b1));
        return cmk<V>(s.x, s.y);
    } else {
        V a0 = cmk<V>(0, 0), a1 = a0;
        int i = 0;
#pragma unroll 1
        for (; i + 1 < n; i += 2) {
            a0 = cfma(t[i], u[i], a0);
            a1 = cfma(t[i + 1], u[i + 1], a1);
        }
        if (i < n) a0 = cfma(t[i], u[i], a0);
        return cadd(a0, a1);
    }
}

constexpr int MAXF = 128;     // faults per shot
// Internal per-shot status: the shot met a truncation that cuts inside a cluster of singular values and
// runs in a one-warp engine, which has no FP64 split; it is re-run by a CTA engine that redoes such splits
// in FP64.  Never reported to the caller.
constexpr int QC_INTERNAL_FP64_RERUN = -100;
constexpr int OPCH = 32;      // program ops staged per step

template <typename R>
struct EngineParams {
    using V = typename VecOf<R>::T;
    const MpsOp* prog;
    uint32_t nops;
    int nq;
    const uint8_t* chan_kind;
    uint32_t nchan;
    const V* g1;  // [G1_COUNT][4]
    const V* g4;  // [G4_COUNT][16]
    const uint64_t* shots;
    uint64_t ntasks;
    unsigned long long* next_task;
    V* mps;               // slot buffers
    uint64_t slot_stride; // elements
    const uint64_t* off;  // site offsets within a slot [nq+1]
    const int* cap;       // bond capacities [nq+1]
    V* scratch;           // per slot: X (global path) then theta copy
    uint64_t scratch_stride;
    uint64_t xg_elems;    // size of the X part of a slot's scratch
    uint32_t x_smem;      // capacity (elements) of the shared-memory X
    uint32_t x_big;       // warp mode: capacity (elements) of the CTA's shared large work area
    int chi_max;          // capacity of every bond in this launch's slot layout
    int chi_trunc;        // the truncation cap (the caller's chi_max, at most the exact bound)
    int defer_capacity;   // 1: a shot that outgrows the capacity is reported but not counted
    int shared_gpu;       // 1: other batches run concurrently (serving): prefer throughput mode
    double cutoff;
    uint32_t k0, k1;
    uint32_t tg[64];
    int32_t weight;
    int reference;        // 1: noiseless reference run writing into `mps` slot 0
    const V* ref;         // reference state
    const uint64_t* ref_off;  // site offsets of the reference state [nq+1]
    int ref_chi;              // largest bond of the reference state
    const int* ref_dims;  // [nq+1]
    double ref_disc;
    double ref_norm;
    int final_center;
    double tau;           // > 0 fixed threshold, else automatic
    int precision;        // QC_C64 / QC_C128
    qc_shot_result* per_shot;
    unsigned long long* counts;  // [3*(wmax+1)]
    int wmax;
    int* ref_status;      // reference run: 0 ok, else index+1 of the bad measurement
    int* ref_chi_out;     // reference run: chi_peak
    int* ref_dims_out;    // reference run: bond dims [nq+1]
    double* ref_disc_out;
    int sweep_cap;
    unsigned long long* phase_cycles;  // optional [8]: SM cycles per phase of the shots, summed
    int use_tc;                // CTA variants: two-site contractions of large theta on the tensor cores
    double* trace_p1;          // optional [ntasks x trace_k]: readout probabilities of each shot
    const uint64_t* trace_pos; // optional: record row of each task (the capacity re-run pass)
    int trace_k;
};

template <typename R>
struct Shared {
    using V = typename VecOf<R>::T;
    V* X;         // [x_smem]
    int* dims;    // [nq+1]
    uint32_t* fch;
    uint8_t* fcode;
    double* red;  // [64]
    MpsOp* ops;   // [OPCH]
    V* pend;      // [nq][4]: single-qubit gates (and fault Paulis) not yet applied to the site
    V* gate;      // [16]: the 4x4 gate of the current two-site update with the pending gates fused
    int* nf;      // fault count of the current shot
    V* big;       // warp mode: the CTA's shared work area for updates too large for X
    int* big_lock;
    unsigned long long* phase;  // [8] cycles per phase of this engine's current shot (thread 0)
    long long* t_mark;          // start of the current phase
    uint64_t* mbar;             // tensor-core completion barrier
    uint32_t* tmem_slot;        // tensor-memory base address written by the allocation
};

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Block-wide sum of a double; every thread gets the result.
// Barriers of an engine: in warp mode (NT = 32) every warp of the CTA runs its own shot, so the
// engine's barriers are warp barriers.
template <int NT> __device__ __forceinline__ void bsync() {
    if (NT == 32) __syncwarp(); else __syncthreads();
}
template <int NT> __device__ __forceinline__ int bsync_or(int v) {
    if (NT == 32) return __any_sync(0xFFFFFFFFu, v);
    return __syncthreads_or(v);
}

// Sum of a double over the engine's threads; every thread gets the result.
template <int NT>
__device__ double block_sum(double v, double* red, int tid) {
    v = warp_sum<double>(v);
    if (NT == 32) return v;
    const int lane = tid & 31, wid = tid >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0;
    if (tid < 32) {
        t = lane < NT / 32 ? red[lane] : 0.0;
        t = warp_sum<double>(t);
        if (lane == 0) red[32] = t;
    }
    __syncthreads();
    return red[32];
}

// Rotation parameters of one Jacobi pair: FP32 uses the hardware reciprocal square root and fast
// division (the rotation only needs c^2 + s^2 = 1 to rounding), FP64 the correctly rounded forms.
__device__ __forceinline__ float rs_sqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rs_sqrt(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fdiv(double a, double b) { return a / b; }

// The engine's dynamic shared memory.  A pointer into it, rebased with as_smem, is one the compiler knows
// to be a shared-memory address: loads and stores through it are 32-bit-addressed LDS / STS instead of
// generic 64-bit accesses (the work areas are reached through pointers that may also point to global
// scratch, which makes them generic).
extern __shared__ __align__(16) unsigned char qc_dsmem[];
template <typename T>
__device__ __forceinline__ T* as_smem(T* p) {
    const size_t off = __cvta_generic_to_shared(p) - __cvta_generic_to_shared(qc_dsmem);
    return reinterpret_cast<T*>(qc_dsmem + off);
}

template <typename R, int NT>
struct Engine {
    using V = typename VecOf<R>::T;
    const EngineParams<R>& P;
    Shared<R>& S;
    V* slot;      // this CTA's site tensors
    V* xg;        // global X
    V* tcopy;     // theta copy
    R* gsig2;     // singular values and their order when the work area is in global memory
    // per-shot state (uniform, kept in registers of every thread, updated identically)
    int status;
    double disc;
    int degen;
    int chi_peak;
    int nupd;
    int64_t abort_op;
    unsigned long long flops;  // algorithmic flops of this shot (integer counts, thread 0)
    int sweeps;
    int gmem_updates;          // two-site updates whose Jacobi matrix lived in global memory
    int resplits;              // complex64 splits redone in FP64 (a cut inside a cluster)

    const int tid_;  // thread index within the engine (the warp lane in warp mode)
    uint64_t task_ = 0;
    uint32_t tmem_ = 0;       // tensor-memory accumulators (CTA variants with use_tc)
    uint32_t tc_parity_ = 0;  // parity of the next completion phase of S.mbar

    __device__ Engine(const EngineParams<R>& p, Shared<R>& s, int slot_id, int tid)
        : P(p), S(s), tid_(tid) {
        slot = P.mps + (uint64_t)slot_id * P.slot_stride;
        xg = P.scratch + (uint64_t)slot_id * P.scratch_stride;
        tcopy = xg + P.xg_elems;
        gsig2 = reinterpret_cast<R*>(tcopy + (size_t)(2 * P.chi_max) * (2 * P.chi_max));
    }

    __device__ V* site(int q) { return slot + P.off[q]; }

    // Phase timing (verification hook): thread 0 charges the SM cycles since the last mark to phase k.
    enum { PH_FAULTS, PH_CONTRACT, PH_JACOBI, PH_SPLIT_OUT, PH_MOVE, PH_PSWAP, PH_READOUT, PH_FINISH };
    __device__ __forceinline__ void tick() {
        if (P.phase_cycles && tid_ == 0) *S.t_mark = clock64();
    }
    __device__ __forceinline__ void tock(int k) {
        if (P.phase_cycles && tid_ == 0) {
            const long long t = clock64();
            S.phase[k] += (unsigned long long)(t - *S.t_mark);
            *S.t_mark = t;
        }
    }

    // ---- single-qubit gates are deferred: pend[q] <- g pend[q] (thread 0 only; consumers start
    //      with a barrier).  A gate on the physical index keeps the canonical form, so it can wait
    //      until the next two-site update or readout of its site, where it is fused.
    __device__ void defer1(int q, V g00, V g01, V g10, V g11) {
        if (tid_ != 0) return;
        V* u = S.pend + q * 4;
        const V u00 = u[0], u01 = u[1], u10 = u[2], u11 = u[3];
        u[0] = cfma(g00, u00, cmul(g01, u10));
        u[1] = cfma(g00, u01, cmul(g01, u11));
        u[2] = cfma(g10, u00, cmul(g11, u10));
        u[3] = cfma(g10, u01, cmul(g11, u11));
    }

    __device__ void defer_pauli(int q, uint32_t p) {
        if (p == 0) return;
        const V z = cmk<V>(0, 0), one = cmk<V>(1, 0), mone = cmk<V>(-1, 0);
        if (p == 1) defer1(q, z, one, one, z);
        else if (p == 2) defer1(q, z, cmk<V>(0, -1), cmk<V>(0, 1), z);
        else defer1(q, one, z, z, mone);
    }

    __device__ void reset_pend(int q) {
        V* u = S.pend + q * 4;
        u[0] = cmk<V>(1, 0); u[1] = cmk<V>(0, 0); u[2] = cmk<V>(0, 0); u[3] = cmk<V>(1, 0);
    }

    // Apply site q's pending gate to its tensor (all threads; ends with a barrier).
    __device__ void flush_site(int q) {
        const V* u = S.pend + q * 4;
        const V g00 = u[0], g01 = u[1], g10 = u[2], g11 = u[3];
        const int cl = S.dims[q], cr = S.dims[q + 1];
        V* a = site(q);
#pragma unroll 1
        for (int e = tid_; e < cl * cr; e += NT) {
            const int l = e / cr, r = e - l * cr;
            V* p0 = a + (l * 2) * cr + r;
            V* p1 = p0 + cr;
            const V x = *p0, y = *p1;
            *p0 = cfma(g00, x, cmul(g01, y));
            *p1 = cfma(g10, x, cmul(g11, y));
        }
        bsync<NT>();
        if (tid_ == 0) reset_pend(q);
        bsync<NT>();
    }

    // Sum over the block in the working precision (identical on every thread).
    __device__ R sum_r(R v) { return sum_rs<R>(v); }
    template <typename RS>
    __device__ RS sum_rs(RS v) {
        if (NT == 32) return warp_sum<RS>(v);
        return (RS)block_sum<NT>((double)v, S.red, tid_);
    }

    // ---- one column pair of the Jacobi sweep -------------------------------------------------------
    // Dot products over this lane's rows i = gl, gl+g, ...: alpha = |a|^2, beta = |b|^2,
    // gamma = a^H b = gr + i gi.  Complex64 uses the paired FP32 FMA (two lanes of one 64-bit
    // register per instruction): the real and imaginary parts accumulate separately and are added
    // at the end.
    template <typename RS>
    __device__ __forceinline__ void pair_dots(const typename VecOf<RS>::T* a, const typename VecOf<RS>::T* b,
                                              int rows, int gl, int g, RS& al, RS& be, RS& gr, RS& gi) {
        using VS = typename VecOf<RS>::T;
        if constexpr (sizeof(RS) == 4) {
            float2 sa = make_float2(0.f, 0.f), sb = sa, sg = sa, sh = sa;
            const float2* pa = a + gl;
            const float2* pb = b + gl;
            const float2* const pe = a + rows;
#pragma unroll 1
            for (; pa < pe; pa += g, pb += g) {  // rows gl, gl + g, ... walked by pointer
                const float2 x = *pa, y = *pb;
                sa = __ffma2_rn(x, x, sa);
                sb = __ffma2_rn(y, y, sb);
                sg = __ffma2_rn(x, y, sg);                            // (x.re y.re, x.im y.im)
                sh = __ffma2_rn(x, make_float2(y.y, y.x), sh);         // (x.re y.im, x.im y.re)
            }
            al = sa.x + sa.y;
            be = sb.x + sb.y;
            gr = sg.x + sg.y;
            gi = sh.x - sh.y;
        } else {
#pragma unroll 1
            for (int i = gl; i < rows; i += g) {
                const VS x = a[i], y = b[i];
                al = fma(x.x, x.x, fma(x.y, x.y, al));
                be = fma(y.x, y.x, fma(y.y, y.y, be));
                gr = fma(x.x, y.x, fma(x.y, y.y, gr));
                gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
            }
        }
    }

    // The rotation of one pair: a <- c a - w b,  b <- conj(w) a + c b,  w = s e^{-i phi} = (wr, wi).
    template <typename RS>
    __device__ __forceinline__ void pair_rotate(typename VecOf<RS>::T* a,
                                                typename VecOf<RS>::T* b, int rows, int gl, int g, RS c,
                                                RS wr, RS wi) {
        using VS = typename VecOf<RS>::T;
        if constexpr (sizeof(RS) == 4) {
            const float2 cc = make_float2(c, c), nw = make_float2(-wr, -wr), ws = make_float2(wi, -wi);
            const float2 wp = make_float2(wr, wr);
            float2* pa = a + gl;
            float2* pb = b + gl;
            float2* const pe = a + rows;
#pragma unroll 1
            for (; pa < pe; pa += g, pb += g) {
                const float2 x = *pa, y = *pb;
                float2 t = __fmul2_rn(nw, y);                          // -w y
                t = __ffma2_rn(ws, make_float2(y.y, y.x), t);
                float2 u = __fmul2_rn(cc, y);                          // conj(w) x + c y
                u = __ffma2_rn(wp, x, u);
                u = __ffma2_rn(ws, make_float2(x.y, x.x), u);
                *pa = __ffma2_rn(cc, x, t);
                *pb = u;
            }
        } else {
#pragma unroll 1
            for (int i = gl; i < rows; i += g) {
                const VS x = a[i], y = b[i];
                const RS wyx = wr * y.x - wi * y.y, wyy = wr * y.y + wi * y.x;  // w y
                const RS vxx = wr * x.x + wi * x.y, vxy = wr * x.y - wi * x.x;  // conj(w) x
                a[i] = cmk<VS>(c * x.x - wyx, c * x.y - wyy);
                b[i] = cmk<VS>(vxx + c * y.x, vxy + c * y.y);
            }
        }
    }

    // ---- one Jacobi rotation of a column pair ------------------------------------------------------
    // The g lanes of a group (gl = lane within the group) form alpha = |a|^2, beta = |b|^2 and
    // gamma = a^H b over the rows and, unless the pair is already orthogonal to the tolerance, rotate
    // it.  Every lane takes part in the shuffles; `act` marks groups that own a pair.  Pairs whose
    // smaller column is below the numerical floor are left alone: such a column is rounding noise of
    // a rank-deficient theta, and rotating it against a large column never reaches relative
    // orthogonality.  Returns 1 when this lane's group rotated.
    template <typename RS>
    __device__ __forceinline__ int pair_step(typename VecOf<RS>::T* a, typename VecOf<RS>::T* b, int rows, int gl,
                                             int g, bool act, RS tol, RS floor2) {
        RS al = 0, be = 0, gr = 0, gi = 0;
        if (act) pair_dots(a, b, rows, gl, g, al, be, gr, gi);
        for (int o = g >> 1; o > 0; o >>= 1) {
            al += __shfl_xor_sync(0xFFFFFFFFu, al, o);
            be += __shfl_xor_sync(0xFFFFFFFFu, be, o);
            gr += __shfl_xor_sync(0xFFFFFFFFu, gr, o);
            gi += __shfl_xor_sync(0xFFFFFFFFu, gi, o);
        }
        const RS g2 = gr * gr + gi * gi;
        if (act && g2 > tol * tol * (al * be) && g2 > (RS)0 && fmin(al, be) > floor2) {
            const RS rg = rs_sqrt(g2);                    // 1 / |gamma|
            const RS zeta = (be - al) * (RS)0.5 * rg;
            const RS t = fdiv(zeta >= 0 ? (RS)1 : (RS)-1, fabs(zeta) + sqrt((RS)1 + zeta * zeta));
            const RS c = rs_sqrt((RS)1 + t * t), sn = c * t;
            pair_rotate(a, b, rows, gl, g, c, sn * gr * rg, -sn * gi * rg);
            return 1;
        }
        return 0;
    }

    // Lane groups for `pairs` concurrent pairs: G groups of g = 32 / G lanes per warp (G a power of
    // two, up to one lane per pair), so that small matrices keep every lane busy and reduce over short
    // shuffle trees.
    __device__ __forceinline__ void lane_groups(int pairs, int rows, int& G, int& g, int& grp, int& gl) const {
        constexpr int NW = NT / 32;
        const int lane = tid_ & 31;
        const int ppw = (pairs + NW - 1) / NW;
        G = 1;
        while (G < ppw && G < 32) G <<= 1;
        g = 32 / G;
        grp = lane / g;
        gl = lane - grp * g;
    }

    template <typename RS>
    __device__ __forceinline__ RS jacobi_tol(int rows) const {
        const RS eps = sizeof(RS) == 4 ? (RS)FLT_EPSILON : (RS)DBL_EPSILON;
        return (RS)4 * eps * sqrt((RS)rows);
    }

    // ---- one-sided Jacobi on the columns of X (rows x cols, cols even, leading dimension ld) -----
    // Round-robin ordering: cols-1 rounds of cols/2 disjoint column pairs, spread over the warps and
    // their lane groups.  In the working precision X is always in shared memory (the split stages a
    // matrix that lives in global memory block by block), so the loops take shared-memory addressing.
    template <typename RS>
    __device__ bool jacobi(typename VecOf<RS>::T* X, int rows, int cols, int ld, RS floor2, int max_sweeps = 0,
                           int* any_rotation = nullptr) {
        if constexpr (sizeof(RS) == sizeof(R)) X = as_smem(X);
        const int wid = tid_ >> 5;
        constexpr int NW = NT / 32;
        const RS tol = jacobi_tol<RS>(rows);
        const int half = cols / 2, cm1 = cols - 1;
        int G, g, grp, gl;
        lane_groups(half, rows, G, g, grp, gl);
        const int cap = max_sweeps > 0 ? max_sweeps : P.sweep_cap;
#pragma unroll 1
        for (int sweep = 0; sweep < cap; ++sweep) {
            int rotated = 0;
#pragma unroll 1
            for (int k = 0; k < cm1; ++k) {
#pragma unroll 1
                for (int base = wid * G; base < half; base += NW * G) {
                    const int pr = base + grp;
                    const bool act = pr < half;
                    const int sa = act ? pr : 0, sb = cols - 1 - sa;
                    // round-robin position -> column: 1 + (s - 1 + k) mod (cols - 1), both terms < cols - 1
                    int ia = sa - 1 + k, ib = sb - 1 + k;
                    ia -= ia >= cm1 ? cm1 : 0;
                    ib -= ib >= cm1 ? cm1 : 0;
                    const int ca = sa == 0 ? 0 : 1 + ia;
                    const int cb = 1 + ib;
                    rotated |= pair_step(X + (size_t)ca * ld, X + (size_t)cb * ld, rows, gl, g, act, tol, floor2);
                }
                bsync<NT>();
            }
            if (max_sweeps == 0) ++sweeps;
            const int any = bsync_or<NT>(rotated);
            if (any && any_rotation) *any_rotation = 1;
            if (!any) return true;
        }
        return max_sweeps > 0;  // an inner pass is not required to converge on its own
    }

    // ---- the cross pairs of two column blocks held side by side in X ------------------------------
    // Columns [0, ni) and [ni, ni + nj).  Round k pairs column i of the smaller block with column
    // (i + k) mod n_l of the larger (n_l columns): each round is a set of disjoint pairs, and n_l
    // rounds visit all ni x nj pairs once.  Returns 1 when this thread's group rotated.
    template <typename RS>
    __device__ __forceinline__ int cross_pass(typename VecOf<RS>::T* X, int rows, int ni, int nj, int ld, RS floor2) {
        const int wid = tid_ >> 5;
        constexpr int NW = NT / 32;
        const RS tol = jacobi_tol<RS>(rows);
        const bool sw = ni > nj;
        const int ns = sw ? nj : ni, nl = sw ? ni : nj;
        const int s0 = sw ? ni : 0, l0 = sw ? 0 : ni;
        int G, g, grp, gl;
        lane_groups(ns, rows, G, g, grp, gl);
        int rotated = 0;
#pragma unroll 1
        for (int k = 0; k < nl; ++k) {
#pragma unroll 1
            for (int base = wid * G; base < ns; base += NW * G) {
                const int i = base + grp;
                const bool act = i < ns;
                const int ii = act ? i : 0;
                int j = ii + k;
                j -= j >= nl ? nl : 0;
                rotated |= pair_step(X + (size_t)(s0 + ii) * ld, X + (size_t)(l0 + j) * ld, rows, gl, g, act, tol,
                                     floor2);
            }
            bsync<NT>();
        }
        return rotated;
    }

    // ---- block Jacobi for an X that lives in global memory ----------------------------------------
    // The columns are cut into blocks of bw (even, or 1 when only two columns fit) that fit twice into
    // the shared work area W.  One outer sweep visits every column pair exactly once, as one cyclic
    // sweep of the plain Jacobi does in another order: the blocks are paired round-robin; each pair is
    // staged into shared memory once, in the first round each block's internal pairs get one
    // round-robin pass, and in every round the staged pair's cross pairs are rotated; then the pair is
    // written back.
    template <typename RS>
    __device__ bool jacobi_blocked(typename VecOf<RS>::T* X, int rows, int cols, int ld, RS floor2,
                                   typename VecOf<RS>::T* W, int bw) {
        W = as_smem(W);
        const int lw = rows + 1;
        const int nb = (cols + bw - 1) / bw;
        const int nbp = nb + (nb & 1);  // an even number of blocks (the last may be a dummy)
#pragma unroll 1
        for (int sweep = 0; sweep < P.sweep_cap; ++sweep) {
            int rot = 0;
#pragma unroll 1
            for (int k = 0; k < nbp - 1; ++k) {
#pragma unroll 1
                for (int pr = 0; pr < nbp / 2; ++pr) {
                    const int sa = pr, sb = nbp - 1 - pr;
                    int ia = sa - 1 + k, ib = sb - 1 + k;
                    ia -= ia >= nbp - 1 ? nbp - 1 : 0;
                    ib -= ib >= nbp - 1 ? nbp - 1 : 0;
                    const int bi = sa == 0 ? 0 : 1 + ia;
                    const int bj = 1 + ib;
                    const int i0 = bi * bw, j0 = bj * bw;
                    const int ni = bi < nb ? min(cols, i0 + bw) - i0 : 0;
                    const int nj = bj < nb ? min(cols, j0 + bw) - j0 : 0;
                    const int nc = ni + nj;
                    if (nc == 0) continue;
#pragma unroll 1
                    for (int e = tid_; e < nc * rows; e += NT) {
                        const int c = e / rows, i = e - c * rows;
                        W[(size_t)c * lw + i] = c < ni ? X[(size_t)(i0 + c) * ld + i] : X[(size_t)(j0 + c - ni) * ld + i];
                    }
                    bsync<NT>();
                    if (k == 0) {  // every block is staged once in the first round: its internal pairs
                        if (ni >= 2) jacobi(W, rows, ni, lw, floor2, 1, &rot);
                        if (nj >= 2) jacobi(W + (size_t)ni * lw, rows, nj, lw, floor2, 1, &rot);
                    }
                    if (ni && nj) rot |= cross_pass(W, rows, ni, nj, lw, floor2);
#pragma unroll 1
                    for (int e = tid_; e < nc * rows; e += NT) {
                        const int c = e / rows, i = e - c * rows;
                        const auto v = W[(size_t)c * lw + i];
                        if (c < ni) X[(size_t)(i0 + c) * ld + i] = v;
                        else X[(size_t)(j0 + c - ni) * ld + i] = v;
                    }
                    bsync<NT>();
                }
            }
            ++sweeps;
            if (!bsync_or<NT>(rot)) return true;
        }
        return false;
    }

    // ---- singular values of the orthogonalised columns: norms, descending order (ties: lower
    //      index first), truncation rule in FP64.  Returns the kept count r; S.red[41] holds the
    //      renormalisation factor.
    template <typename RS>
    __device__ int spectrum(typename VecOf<RS>::T* X, int rows, int cols, int ld, RS* sig2, int* perm, RS floor2) {
        // singular values: column norms, then descending order (ties: lower index first)
        {
            const int lane = tid_ & 31, wid = tid_ >> 5;
            constexpr int NW = NT / 32;
            const int cpw = (cols + NW - 1) / NW;
            int G = 1;
            while (G < cpw && G < 32) G <<= 1;
            const int g = 32 / G, grp = lane / g, gl = lane - grp * g;
#pragma unroll 1
            for (int base = wid * G; base < cols; base += NW * G) {
                const int j = base + grp;
                RS sq = 0;
                if (j < cols) {
                    const auto* col = X + (size_t)j * ld;
#pragma unroll 1
                    for (int i = gl; i < rows; i += g) sq = fma(col[i].x, col[i].x, fma(col[i].y, col[i].y, sq));
                }
                for (int o = g >> 1; o > 0; o >>= 1) sq += __shfl_xor_sync(0xFFFFFFFFu, sq, o);
                if (j < cols && gl == 0) sig2[j] = sq;
            }
        }
        bsync<NT>();
#pragma unroll 1
        for (int j = tid_; j < cols; j += NT) {
            const RS sj = sig2[j];
            int rk = 0;
#pragma unroll 1
            for (int k = 0; k < cols; ++k) {
                const RS sk = sig2[k];
                rk += (sk > sj) || (sk == sj && k < j);
            }
            perm[rk] = j;
        }
        bsync<NT>();
        // truncation rule, FP64: smallest r >= 1 with discarded tail <= cutoff * total, r <= chi_max.
        // The first warp works on the sorted values in contiguous chunks, one per lane: chunk sums,
        // a suffix scan over the lanes, then every position k >= 1 whose tail sum_{k' >= k} s_k'^2
        // exceeds the threshold is counted (the tail shrinks with k, so those positions are
        // 1 .. r-1).
        if (tid_ < 32) {
            const unsigned full = 0xFFFFFFFFu;
            const int lane = tid_;
            const int c = (cols + 31) >> 5;
            const int k0 = min(cols, lane * c), k1 = min(cols, k0 + c);
            double loc = 0;
            int nzl = 0;
#pragma unroll 1
            for (int k = k0; k < k1; ++k) {
                const RS v = sig2[perm[k]];
                loc += (double)v;
                nzl += v > floor2;
            }
            double incl = loc;  // sum of this lane's chunk and every later one
            for (int o = 1; o < 32; o <<= 1) {
                const double t = __shfl_down_sync(full, incl, o);
                if (lane + o < 32) incl += t;
            }
            const double tot = __shfl_sync(full, incl, 0);
            double after = __shfl_down_sync(full, incl, 1);
            if (lane == 31) after = 0;
            const int nz = __reduce_add_sync(full, nzl);
            const double thr = P.cutoff * tot;
            int cnt = 0;
            double tail = after;
#pragma unroll 1
            for (int k = k1 - 1; k >= k0; --k) {
                tail += (double)sig2[perm[k]];
                cnt += (k >= 1 && tail > thr);
            }
            int r = 1 + __reduce_add_sync(full, cnt);
            r = min(r, P.chi_trunc);
            r = min(r, max(nz, 1));
            // dropped = the tail sum from position r: the lane whose chunk holds r adds its chunk's part
            // to the sum of the later chunks; kept = total - dropped
            double tr = after;
#pragma unroll 1
            for (int k = k1 - 1; k >= k0 && k >= r; --k) tr += (double)sig2[perm[k]];
            const double dropped = r < cols ? __shfl_sync(full, tr, min(31, r / c)) : 0.0;
            const double kept = tot - dropped;
            if (lane == 0) {
                int dg = 0;
                // a cut inside a cluster: the last kept and the first dropped value agree to what the
                // working precision resolves (FP64: s_{r-1} / s_r - 1 < 1e-8, i.e. 2e-8 on the squares;
                // FP32: the Jacobi stops at |a^H b| <= 4 eps sqrt(rows) |a||b|, so squared norms closer
                // than 32 eps sqrt(rows) relative are not told apart); a dropped value at the numerical
                // floor is not a cluster member
                // FP32 also needs the dropped value to carry more than the cutoff's share of the weight
                // (a cut set by chi_max): a cut the cutoff makes among tiny near-equal values at the
                // FP32 noise level drops at most cutoff x total whichever of them it keeps
                if (r < cols) {
                    const double a2 = (double)sig2[perm[r - 1]], b2 = (double)sig2[perm[r]];
                    const double rel = sizeof(RS) == 8 ? 2e-8 + 1e-16 : 32.0 * FLT_EPSILON * (double)sqrtf((float)rows);
                    const double sig = sizeof(RS) == 8 ? (double)floor2 : fmax((double)floor2, P.cutoff * tot);
                    dg = b2 > sig && a2 <= b2 * (1.0 + rel);
                }
                S.red[40] = tot > 0 ? dropped / tot : 0.0;
                S.red[41] = kept > 0 ? rsqrt(kept) : 0.0;  // applied in the working precision
                S.red[42] = (double)r;
                S.red[43] = (double)dg;
            }
        }
        bsync<NT>();
        const int r = (int)S.red[42];
        disc += S.red[40];
        degen += (int)S.red[43];
        return r;
    }

    __device__ void release_big(bool locked) {
        if (!locked) return;
        bsync<NT>();
        if (tid_ == 0) {
            __threadfence_block();
            atomicExch(S.big_lock, 0);
        }
    }

    // ---- two-site update on (q, q+1) -----------------------------------------------------------
    // The single-qubit gates pending on both sites are fused into the 4x4 gate, then the pair is split.
    // On the complex64 path a split whose truncation cuts inside a cluster of equal singular values
    // (the last kept and the first dropped value agree to what FP32 resolves, and the dropped value is
    // above the numerical floor) is redone in FP64 from the unchanged site tensors: contraction,
    // Jacobi, spectrum and truncation rule in FP64, the factors stored back in complex64.
    __device__ void update(int q, const V* g, bool right) {
        bsync<NT>();  // pending gates written by thread 0, dims of the previous update
        tick();
        // fused gate: gate[(a,b),(s',t')] = sum_{s,t} g[(a,b),(s,t)] U_q[s,s'] U_{q+1}[t,t']
        if (tid_ < 16) {
            const int abi = tid_ >> 2, sp = (tid_ >> 1) & 1, tp = tid_ & 1;
            const V* uq = S.pend + q * 4;
            const V* ur = S.pend + (q + 1) * 4;
            V acc = cmk<V>(0, 0);
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                const V w = cmul(uq[(st >> 1) * 2 + sp], ur[(st & 1) * 2 + tp]);
                acc = cfma(g[abi * 4 + st], w, acc);
            }
            S.gate[tid_] = acc;
        }
        bsync<NT>();
        if (tid_ == 0) { reset_pend(q); reset_pend(q + 1); }
        if constexpr (sizeof(R) == 4) {
            if (split<float>(q, right) == SPLIT_REDO_FP64) {
                if constexpr (NT == 32) {
                    // the warp engine stays lean (no FP64 split in its code): the shot is re-run by a CTA
                    status = QC_INTERNAL_FP64_RERUN;
                } else {
                    ++resplits;
                    split<double>(q, right);
                }
            }
        } else {
            split<double>(q, right);
        }
    }

    // ---- theta' = gate (A B) on the tensor cores (CTA variants, theta in global memory) -------------
    // The complex product takes three real products (P1 = Ar Br, P2 = Ai Bi, P3 = (Ar+Ai)(Br+Bi);
    // Re = P1 - P2, Im = P3 - P1 - P2), each as three TF32 MMAs on hi/lo splits of the operands (about
    // FP32 accuracy).  Output tiles of 128 rows (l, s') x 32 columns: 16 values of r for t' = 0 and the
    // same 16 for t' = 1, so that the 4x4 gate can be applied in the epilogue (the two rows s' of one l
    // sit in adjacent lanes).  K in chunks of 16: the six A and six B operand components are staged in
    // the engine's shared work area in the K-major no-swizzle layout (60 KB), one thread issues 18 MMAs
    // into three tensor-memory accumulators of 32 columns and commits them to an mbarrier, every thread
    // waits (bounded), and the next chunk is staged.  Writes X and T as the CUDA-core contraction does
    // and accumulates |theta'|^2 into fro.  Returns false when a wait ran out (the shot then ends with
    // QC_ETIMEOUT).
    __device__ bool tc_contract(const V* A, const V* B, int m, int n, int cr, int cm, V* X, V* T, int ld, bool xt,
                                R& fro) {
        constexpr int KC = 16, TA = 128 * KC, TB = 32 * KC;
        float* sa = reinterpret_cast<float*>(((uintptr_t)S.X + 1023) & ~(uintptr_t)1023);
        float* sb = sa + 6 * TA;
        const uint32_t idesc = tc::idesc_tf32(128, 32);
        const int warp = tid_ >> 5, lane = tid_ & 31, quarter = warp & 3, wgrp = warp >> 2;
        const V* gt = S.gate;
#pragma unroll 1
        for (int mt = 0; mt < m; mt += 128) {
#pragma unroll 1
            for (int r0 = 0; r0 < cr; r0 += 16) {
#pragma unroll 1
                for (int kc = 0; kc < cm; kc += KC) {
#pragma unroll 1
                    for (int e = tid_; e < TA; e += NT) {  // A rows mt.., K kc..
                        const int rr = e / KC, kk = e - rr * KC;
                        const int i = mt + rr, k = kc + kk;
                        const V a = (i < m && k < cm) ? A[(size_t)i * cm + k] : cmk<V>(0, 0);
                        float h, l;
                        const uint32_t o = tc::kmaj_off(rr, kk, KC) >> 2;
                        tc::split_tf32(a.x, h, l); sa[0 * TA + o] = h; sa[1 * TA + o] = l;
                        tc::split_tf32(a.y, h, l); sa[2 * TA + o] = h; sa[3 * TA + o] = l;
                        tc::split_tf32(a.x + a.y, h, l); sa[4 * TA + o] = h; sa[5 * TA + o] = l;
                    }
#pragma unroll 1
                    for (int e = tid_; e < TB; e += NT) {  // B columns (t', r0 + jj), K kc..
                        const int jj = e / KC, kk = e - jj * KC;
                        const int r = r0 + (jj & 15), tp = jj >> 4, k = kc + kk;
                        const V b = (r < cr && k < cm) ? B[(size_t)k * n + tp * cr + r] : cmk<V>(0, 0);
                        float h, l;
                        const uint32_t o = tc::kmaj_off(jj, kk, KC) >> 2;
                        tc::split_tf32(b.x, h, l); sb[0 * TB + o] = h; sb[1 * TB + o] = l;
                        tc::split_tf32(b.y, h, l); sb[2 * TB + o] = h; sb[3 * TB + o] = l;
                        tc::split_tf32(b.x + b.y, h, l); sb[4 * TB + o] = h; sb[5 * TB + o] = l;
                    }
                    tc::fence_async_smem();
                    tc::fence_before_sync();
                    bsync<NT>();
                    tc::fence_after_sync();
                    if (tid_ == 0) {
                        const uint32_t a0 = tc::smem_u32(sa), b0 = tc::smem_u32(sb);
                        constexpr uint32_t sbo = (KC / 4) * 128;
#pragma unroll
                        for (int ks = 0; ks < KC / 8; ++ks) {
                            const uint32_t ko = ks * 256;
                            const uint32_t first = (kc > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                            for (int pr = 0; pr < 3; ++pr) {  // P1 (re, re), P2 (im, im), P3 (sum, sum)
                                const uint32_t d = tmem_ + 32u * pr;
                                const uint64_t ah = tc::smem_desc(a0 + (2 * pr) * TA * 4 + ko, 128, sbo);
                                const uint64_t al = tc::smem_desc(a0 + (2 * pr + 1) * TA * 4 + ko, 128, sbo);
                                const uint64_t bh = tc::smem_desc(b0 + (2 * pr) * TB * 4 + ko, 128, sbo);
                                const uint64_t bl = tc::smem_desc(b0 + (2 * pr + 1) * TB * 4 + ko, 128, sbo);
                                tc::mma_tf32(d, ah, bh, idesc, first);
                                tc::mma_tf32(d, ah, bl, idesc, 1u);
                                tc::mma_tf32(d, al, bh, idesc, 1u);
                            }
                        }
                        tc::mma_commit(S.mbar);
                    }
                    const bool ok = tc::mbar_wait(S.mbar, tc_parity_, 1 << 24);
                    tc_parity_ ^= 1u;
                    tc::fence_after_sync();
                    if (bsync_or<NT>(!ok)) return false;
                }
                // epilogue: this thread's row i = (l, s'); column pieces p of 8 values of r
                const int i = mt + quarter * 32 + lane;
                const uint32_t ta = tmem_ + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
                for (int pc = wgrp; pc < 2; pc += NT / 128) {
                    float p1a[8], p2a[8], p3a[8], p1b[8], p2b[8], p3b[8];
                    tc::tmem_ld8(ta + 0 + pc * 8, p1a);
                    tc::tmem_ld8(ta + 32 + pc * 8, p2a);
                    tc::tmem_ld8(ta + 64 + pc * 8, p3a);
                    tc::tmem_ld8(ta + 16 + pc * 8, p1b);
                    tc::tmem_ld8(ta + 48 + pc * 8, p2b);
                    tc::tmem_ld8(ta + 80 + pc * 8, p3b);
#pragma unroll
                    for (int c = 0; c < 8; ++c) {
                        const V th0 = cmk<V>(p1a[c] - p2a[c], p3a[c] - p1a[c] - p2a[c]);  // theta[(l,s'),(0,r)]
                        const V th1 = cmk<V>(p1b[c] - p2b[c], p3b[c] - p1b[c] - p2b[c]);  // theta[(l,s'),(1,r)]
                        const V o0 = cmk<V>(__shfl_xor_sync(0xFFFFFFFFu, th0.x, 1), __shfl_xor_sync(0xFFFFFFFFu, th0.y, 1));
                        const V o1 = cmk<V>(__shfl_xor_sync(0xFFFFFFFFu, th1.x, 1), __shfl_xor_sync(0xFFFFFFFFu, th1.y, 1));
                        const int sp = i & 1;
                        // th[u], u = 2 s' + t'
                        const V t0 = sp ? o0 : th0, t1 = sp ? o1 : th1, t2 = sp ? th0 : o0, t3 = sp ? th1 : o1;
                        const int r = r0 + pc * 8 + c;
                        if (i < m && r < cr) {
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                const int st = 2 * sp + t;
                                V v = cmul(gt[st * 4 + 0], t0);
                                v = cfma(gt[st * 4 + 1], t1, v);
                                v = cfma(gt[st * 4 + 2], t2, v);
                                v = cfma(gt[st * 4 + 3], t3, v);
                                const int j = t * cr + r;
                                fro = fma(v.x, v.x, fma(v.y, v.y, fro));
                                T[(size_t)i * n + j] = v;
                                if (xt) X[(size_t)j * ld + i] = v;
                                else X[(size_t)i * ld + j] = cmk<V>(v.x, -v.y);
                            }
                        }
                    }
                }
                tc::fence_before_sync();
                bsync<NT>();  // accumulators read before the next tile's MMAs overwrite them
                tc::fence_after_sync();
            }
        }
        return true;
    }

    enum { SPLIT_DONE = 0, SPLIT_FAIL = 1, SPLIT_REDO_FP64 = 2 };

    template <typename VS>
    __device__ __forceinline__ static VS widen(const V& x) { return cmk<VS>(x.x, x.y); }

    // Split of the pair (q, q+1) in precision RS (R, or double for the FP64 re-split of a complex64 state).
    // Work area, per update: X (Jacobi matrix, ld x cols) | T (theta' copy, m x n; A and B are staged here
    // first and read by the contraction, theta' is copied in afterwards) | sig2 | perm, in shared memory
    // when it fits; otherwise X (if needed) and T go to the slot's global scratch and A, B are read from
    // the site tensors.  The FP64 re-split always works in the global scratch (sized for it).
    template <typename RS>
    __device__ int split(int q, bool right) {
        using VS = typename VecOf<RS>::T;
        constexpr bool promoted = sizeof(RS) > sizeof(R);
        const int cl = S.dims[q], cm = S.dims[q + 1], cr = S.dims[q + 2];
        const int m = 2 * cl, n = 2 * cr;
        // the Jacobi orthogonalises the columns of theta' (xt) or of theta'^H, whichever has fewer
        // (cost ~ rows x cols^2); a square theta' follows the centre's direction
        const bool xt = n < m || (n == m && right);
        const int rows = xt ? m : n, cols = xt ? n : m;
        const int ld = rows + 1;
        const uint64_t ab = (uint64_t)m * cm + (uint64_t)cm * n;
        const uint64_t treg = max((uint64_t)m * n, ab);
        const uint64_t sgw = ((uint64_t)cols * (sizeof(R) + sizeof(int)) + sizeof(V) - 1) / sizeof(V);
        const uint64_t need = (uint64_t)ld * cols + treg + sgw;
        bool fast = !promoted && need <= P.x_smem;
        V* W = S.X;
        bool locked = false;
        if (!promoted && !fast && NT == 32 && need <= P.x_big) {
            // warp mode: borrow the CTA's large work area (bounded wait; the global path otherwise)
            int got = 0;
            if (tid_ == 0) {
#pragma unroll 1
                for (int it = 0; it < (1 << 22); ++it) {
                    if (atomicCAS(S.big_lock, 0, 1) == 0) { got = 1; break; }
                    __nanosleep(256);
                }
                __threadfence_block();
            }
            got = __shfl_sync(0xFFFFFFFFu, got, 0);
            if (got) { W = S.big; fast = true; locked = true; }
        }
        VS* X;
        VS* T;
        RS* sig2;
        if (promoted) {  // the doubled global scratch: X | theta' | spectrum, all in FP64
            const size_t c2 = (size_t)(2 * P.chi_max);
            X = reinterpret_cast<VS*>(xg);
            T = X + (c2 + 1) * c2;
            sig2 = reinterpret_cast<RS*>(T + c2 * c2);
        } else {
            X = reinterpret_cast<VS*>(fast ? W : ((uint64_t)ld * cols <= P.x_smem ? S.X : xg));
            T = reinterpret_cast<VS*>(fast ? W + (size_t)ld * cols : tcopy);
            sig2 = reinterpret_cast<RS*>(fast ? reinterpret_cast<R*>(W + (size_t)ld * cols + treg) : gsig2);
        }
        int* perm = reinterpret_cast<int*>(sig2 + cols);
        const V* A = site(q);
        const V* B = site(q + 1);
        if (fast) {
            V* As = W + (size_t)ld * cols;
            V* Bs = As + (size_t)m * cm;
#pragma unroll 1
            for (int e = tid_; e < m * cm; e += NT) As[e] = A[e];
#pragma unroll 1
            for (int e = tid_; e < cm * n; e += NT) Bs[e] = B[e];
            A = As;
            B = Bs;
        }
        bsync<NT>();
        const V* gt = S.gate;
        // theta'[(l,s),(t,r)] = sum_{s',t'} gate[(s,t),(s',t')] sum_k A[l,s',k] B[k,t',r]
        RS fro = 0;  // only sets the numerical floor: the working precision suffices
        bool on_tc = false;
        if constexpr (NT >= 128 && sizeof(RS) == 4) {
            // large theta of a CTA variant whose Jacobi matrix lives in global memory: the shared work
            // area is free for the operand tiles (60 KB + alignment)
            on_tc = P.use_tc && !fast && (void*)X == (void*)xg && m >= 64 && cr >= 8 && cm >= 8 &&
                    (uint64_t)P.x_smem * sizeof(V) >= 62 * 1024;
            if (on_tc && !tc_contract(A, B, m, n, cr, cm, reinterpret_cast<V*>(X), reinterpret_cast<V*>(T), ld, xt,
                                      fro)) {
                status = QC_ETIMEOUT;
                release_big(locked);
                return SPLIT_FAIL;
            }
        }
#pragma unroll 1
        for (int e = on_tc ? cl * cr : tid_; e < cl * cr; e += NT) {
            const int l = e / cr, r = e - l * cr;
            VS th[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) th[u] = cmk<VS>(0, 0);
            const V* a0 = A + (l * 2) * cm;
            const V* a1 = a0 + cm;
            if constexpr (sizeof(RS) == 4) {  // complex MACs as two paired FP32 FMAs each
                float2 t0 = make_float2(0.f, 0.f), t1 = t0, t2 = t0, t3 = t0;
                const V* bk = B + r;  // B[k, t', r] walked by pointer (one add per k instead of index products)
#pragma unroll 1
                for (int k = 0; k < cm; ++k, bk += n) {
                    const float2 x0 = a0[k], x1 = a1[k];
                    const float2 y0 = bk[0], y1 = bk[cr];
                    const float2 x0r = make_float2(x0.x, x0.x), x0i = make_float2(-x0.y, x0.y);
                    const float2 x1r = make_float2(x1.x, x1.x), x1i = make_float2(-x1.y, x1.y);
                    const float2 y0s = make_float2(y0.y, y0.x), y1s = make_float2(y1.y, y1.x);
                    t0 = __ffma2_rn(x0i, y0s, __ffma2_rn(x0r, y0, t0));
                    t1 = __ffma2_rn(x0i, y1s, __ffma2_rn(x0r, y1, t1));
                    t2 = __ffma2_rn(x1i, y0s, __ffma2_rn(x1r, y0, t2));
                    t3 = __ffma2_rn(x1i, y1s, __ffma2_rn(x1r, y1, t3));
                }
                th[0] = t0; th[1] = t1; th[2] = t2; th[3] = t3;
            } else {
#pragma unroll 1
                for (int k = 0; k < cm; ++k) {
                    const VS x0 = widen<VS>(a0[k]), x1 = widen<VS>(a1[k]);
                    const VS y0 = widen<VS>(B[(size_t)k * n + r]), y1 = widen<VS>(B[(size_t)k * n + cr + r]);
                    th[0] = cfma(x0, y0, th[0]);
                    th[1] = cfma(x0, y1, th[1]);
                    th[2] = cfma(x1, y0, th[2]);
                    th[3] = cfma(x1, y1, th[3]);
                }
            }
#pragma unroll
            for (int st = 0; st < 4; ++st) {
                VS v = cmk<VS>(0, 0);
#pragma unroll
                for (int u = 0; u < 4; ++u) v = cfma(widen<VS>(gt[st * 4 + u]), th[u], v);
                const int i = l * 2 + (st >> 1), j = (st & 1) * cr + r;
                fro = fma(v.x, v.x, fma(v.y, v.y, fro));
                if (!fast) T[(size_t)i * n + j] = v;
                if (xt) X[(size_t)j * ld + i] = v;
                else X[(size_t)i * ld + j] = cmk<VS>(v.x, -v.y);
            }
        }
        if (fast) {  // A and B are consumed: keep theta' in T for the projection after the split
            bsync<NT>();
#pragma unroll 1
            for (int e = tid_; e < m * n; e += NT) {
                const int i = e / n, j = e - i * n;
                const VS v = xt ? X[(size_t)j * ld + i] : X[(size_t)i * ld + j];
                T[e] = xt ? v : cmk<VS>(v.x, -v.y);
            }
        }
        const double frod = (double)sum_rs<RS>(fro);  // sets the numerical floor only: working precision
        const RS eps = sizeof(RS) == 4 ? (RS)FLT_EPSILON : (RS)DBL_EPSILON;
        const RS fl = (RS)4 * eps * sqrt((RS)rows);
        const RS floor2 = fl * fl * (RS)frod;
        // the blocked Jacobi stages column blocks in the engine's shared work area
        const uint32_t w_cap = (uint32_t)((uint64_t)P.x_smem * sizeof(V) / sizeof(VS));
        // blocks of bw columns, two staged at a time: even (every block pairs up inside) unless only two
        // single columns fit, where the blocked sweep is the plain round-robin one staged pair by pair
        int bw = (int)(w_cap / (2 * (uint32_t)(rows + 1)));
        if (bw >= 2) bw &= ~1;
        const bool in_global = promoted || (void*)X == (void*)xg;
        // an X in global memory always goes through the blocked Jacobi (staged in shared memory), in the
        // working precision the only one there is; the FP64 re-split may run the plain one on global memory
        const bool blocked = in_global && bw >= 1;
        if (in_global && !blocked && !promoted) {
            status = QC_ECAPACITY;  // two columns of X do not fit the work area
            release_big(locked);
            return SPLIT_FAIL;
        }
        gmem_updates += in_global ? 1 : 0;
        tock(PH_CONTRACT);
        if (!(blocked ? jacobi_blocked<RS>(X, rows, cols, ld, floor2, reinterpret_cast<VS*>(S.X), bw)
                      : jacobi<RS>(X, rows, cols, ld, floor2))) {
            status = QC_ENOCONV;
            release_big(locked);
            return SPLIT_FAIL;
        }
        tock(PH_JACOBI);
        const int r = spectrum<RS>(X, rows, cols, ld, sig2, perm, floor2);
        if (!promoted && sizeof(R) == 4 && S.red[43] != 0.0) {
            // a cut inside a cluster: undo this split's statistics and redo it in FP64
            disc -= S.red[40];
            degen -= (int)S.red[43];
            release_big(locked);
            bsync<NT>();
            return SPLIT_REDO_FP64;
        }
        const RS scale = (RS)S.red[41];
        if (r > P.cap[q + 1]) {
            status = QC_ECAPACITY;
            release_big(locked);
            return SPLIT_FAIL;
        }
        // the kept singular values, once per column: sig2[j] <- sqrt(sig2[j])
#pragma unroll 1
        for (int k = tid_; k < r; k += NT) {
            const int j = perm[k];
            const RS sg = sig2[j];
            sig2[j] = sg > (RS)0 ? sqrt(sg) : (RS)0;
        }
        bsync<NT>();
        // normalise the kept columns to unit length (the orthonormal factor)
#pragma unroll 1
        for (int e = tid_; e < r * rows; e += NT) {
            const int k = e / rows, i = e - k * rows;
            const int j = perm[k];
            const RS sv = sig2[j];
            const RS inv = sv > (RS)0 ? fdiv((RS)1, sv) : (RS)0;
            VS* col = X + (size_t)j * ld;
            col[i] = cmk<VS>(col[i].x * inv, col[i].y * inv);
        }
        bsync<NT>();
        V* As = site(q);
        V* Bs = site(q + 1);
        // The factors, in one pair of loops for the four cases (orthogonalised side xt = theta' or its
        // conjugate transpose; centre to the right or the left):
        //   xt,  right: A[q] = U (cl, 2, r);             A[q+1] = scale * U^H theta' (r, 2, cr)
        //   xt,  left:  A[q] = scale * U S (cl, 2, r);   A[q+1] = V^H = S^-1 U^H theta' (r, 2, cr)
        //   !xt, left:  A[q+1] = U'^H (r, 2, cr);         A[q] = scale * theta' U' (cl, 2, r)
        //   !xt, right: A[q+1] = scale * S U'^H (r, 2, cr); A[q] = V' = theta' U' S^-1 (cl, 2, r)
        // (U, U' = the normalised kept columns of X; theta' = V' S U'^H in the !xt cases.)
        {
            const bool plain = xt == right;         // the orthonormal factor unscaled, the projection x scale
            V* Fo = xt ? As : Bs;                   // orthonormal factor: U (m x r) or U'^H (r x n)
            V* Fp = xt ? Bs : As;                   // projection: U^H theta' (r x n) or theta' U' (m x r)
            const int no = xt ? m * r : r * n, dio = xt ? r : n;
#pragma unroll 1
            for (int e = tid_; e < no; e += NT) {
                const int a = e / dio, b = e - a * dio;
                const int k = xt ? b : a, i = xt ? a : b;  // kept index, row of X
                const RS f = plain ? (RS)1 : scale * sig2[perm[k]];
                const VS u = X[(size_t)perm[k] * ld + i];
                Fo[e] = cmk<V>(u.x * f, (xt ? u.y : -u.y) * f);
            }
            const int np = xt ? r * n : m * r, dip = xt ? n : r;
#pragma unroll 1
            for (int e = tid_; e < np; e += NT) {
                const int a = e / dip, b = e - a * dip;
                const int k = xt ? a : b, j = xt ? b : a;  // kept index, other index of theta'
                const VS acc = xt ? dot_conj(X + (size_t)perm[k] * ld, T + j, (size_t)n, m)
                                  : dot_plain(T + (size_t)j * n, X + (size_t)perm[k] * ld, n);
                RS f = scale;
                if (!plain) {
                    const RS svk = sig2[perm[k]];
                    f = svk > (RS)0 ? fdiv((RS)1, svk) : (RS)0;
                }
                Fp[e] = cmk<V>(acc.x * f, acc.y * f);
            }
        }
        bsync<NT>();
        release_big(locked);
        if (tid_ == 0) S.dims[q + 1] = r;
        bsync<NT>();
        tock(PH_SPLIT_OUT);
        chi_peak = max(chi_peak, r);
        ++nupd;
        if (tid_ == 0) {  // integer accounting: the FP64 pipe is narrow on this part
            const unsigned long long M = max(m, n), Nn = min(m, n);
            flops += 8ull * m * cm * n + 128ull * cl * cr + 4ull * (4ull * M * M * Nn + 22ull * Nn * Nn * Nn) +
                     8ull * r * m * n;
        }
        return SPLIT_DONE;
    }

    // ---- QR of X (rows x cols, leading dimension ld) by classical Gram-Schmidt -------------------
    // Each column is orthogonalised against the kept ones, the pass repeated while it removes more
    // than half of the column's squared norm (the Daniel-Gragg-Kaufman-Stewart test), so every kept
    // column is orthogonal to the earlier ones to rounding.  A column whose remainder falls to the
    // floor depends on the kept ones and is dropped.  On return columns 0..k-1 of X hold the
    // orthonormal kept columns in order (the i-th came from column perm[i]), and Rm (row-major,
    // k x cols, zeroed by the caller) holds R: X_in = Q R.  hb: scratch of cols elements.  Returns k.
    __device__ int gram_schmidt(V* X, int rows, int cols, int ld, V* Rm, V* hb, int* perm, R floor2,
                                double& dropped) {
        int k = 0;
#pragma unroll 1
        for (int j = 0; j < cols; ++j) {
            V* x = X + (size_t)j * ld;
            R part = 0;
#pragma unroll 1
            for (int i = tid_; i < rows; i += NT) part = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, part));
            R nold = sum_r(part), nnow = nold;
#pragma unroll 1
            for (int pass = 0; pass < 4 && k > 0; ++pass) {
                {  // h_i = <q_i, x>: the k dot products spread over lane groups (short chains)
                    const int wid = tid_ >> 5;
                    constexpr int NW = NT / 32;
                    int G, g, grp, gl;
                    lane_groups(k, rows, G, g, grp, gl);
#pragma unroll 1
                    for (int base = wid * G; base < k; base += NW * G) {
                        const int i = base + grp;
                        const bool act = i < k;
                        const V* qi = X + (size_t)(act ? i : 0) * ld;
                        R hr = 0, hi = 0;
                        if (act) {
                            if constexpr (sizeof(R) == 4) {  // paired FP32 FMAs, as in the Jacobi
                                float2 s1 = make_float2(0.f, 0.f), s2 = s1;
                                const float2* pq = qi + gl;
                                const float2* px = x + gl;
                                const float2* const pe = qi + rows;
#pragma unroll 1
                                for (; pq < pe; pq += g, px += g) {
                                    const float2 u0 = *pq, x0 = *px;
                                    s1 = __ffma2_rn(u0, x0, s1);                          // (q.re x.re, q.im x.im)
                                    s2 = __ffma2_rn(u0, make_float2(x0.y, x0.x), s2);     // (q.re x.im, q.im x.re)
                                }
                                hr = s1.x + s1.y;
                                hi = s2.x - s2.y;
                            } else {
#pragma unroll 1
                                for (int t = gl; t < rows; t += g) {
                                    hr = fma(qi[t].x, x[t].x, fma(qi[t].y, x[t].y, hr));
                                    hi = fma(qi[t].x, x[t].y, fma(-qi[t].y, x[t].x, hi));
                                }
                            }
                        }
                        for (int o = g >> 1; o > 0; o >>= 1) {
                            hr += __shfl_xor_sync(0xFFFFFFFFu, hr, o);
                            hi += __shfl_xor_sync(0xFFFFFFFFu, hi, o);
                        }
                        if (act && gl == 0) {
                            hb[i] = cmk<V>(hr, hi);
                            V& rr = Rm[(size_t)i * cols + j];
                            rr = cmk<V>(rr.x + hr, rr.y + hi);
                        }
                    }
                }
                bsync<NT>();
                part = 0;
#pragma unroll 1
                for (int t = tid_; t < rows; t += NT) {  // x -= sum_i h_i q_i (two partial sums)
                    V acc = x[t], acc1 = cmk<V>(0, 0);
                    int i = 0;
                    const V* qt = X + t;  // row t of the kept columns 0, 1, ... (stored in order)
#pragma unroll 1
                    for (; i + 1 < k; i += 2, qt += 2 * ld) {
                        const V h = hb[i], u = qt[0];
                        const V h1 = hb[i + 1], u1 = qt[ld];
                        acc = cmk<V>(acc.x - (h.x * u.x - h.y * u.y), acc.y - (h.x * u.y + h.y * u.x));
                        acc1 = cmk<V>(acc1.x + (h1.x * u1.x - h1.y * u1.y), acc1.y + (h1.x * u1.y + h1.y * u1.x));
                    }
                    if (i < k) {
                        const V h = hb[i], u = qt[0];
                        acc = cmk<V>(acc.x - (h.x * u.x - h.y * u.y), acc.y - (h.x * u.y + h.y * u.x));
                    }
                    acc = cmk<V>(acc.x - acc1.x, acc.y - acc1.y);
                    x[t] = acc;
                    part = fma(acc.x, acc.x, fma(acc.y, acc.y, part));
                }
                bsync<NT>();
                nnow = sum_r(part);
                const bool done = nnow > (R)0.5 * nold;
                nold = nnow;
                if (done) break;
            }
            if (nnow > floor2) {
                // the k-th kept column is stored normalised in column k (k <= j; columns k .. j-1 hold
                // nothing that is still needed), so the kept columns stay contiguous
                const R nr = sqrt(nnow), inv = (R)1 / nr;
                V* xk = X + (size_t)k * ld;
#pragma unroll 1
                for (int t = tid_; t < rows; t += NT) xk[t] = cmk<V>(x[t].x * inv, x[t].y * inv);
                if (tid_ == 0) {
                    Rm[(size_t)k * cols + j] = cmk<V>(nr, (R)0);
                    perm[k] = j;
                }
                ++k;
            } else {
                dropped += (double)nnow;
            }
            bsync<NT>();
        }
        return k;
    }

    // ---- centre move between q and q+1 without a gate: QR of one site tensor ---------------------
    // Right: A[q] (m x cm) = Q R, A[q] = Q and the centre R A[q+1].  Left: the same on A[q+1]^H
    // (n x cm); A[q+1] = R^H Q^H gives A[q+1] = Q^H and the centre A[q] R^H.  Columns at the
    // numerical floor are dropped (gram_schmidt), so the bond shrinks to the numerical rank.
    // Nothing else is truncated, so a move leaves the state as it was (Sec. 3.1: moving the
    // orthogonality centre is a gauge change).
    __device__ void move(int q, bool right) {
        bsync<NT>();
        tick();
        const int cl = S.dims[q], cm = S.dims[q + 1], cr = S.dims[q + 2];
        const int m = 2 * cl, n = 2 * cr;
        const int rows = right ? m : n;
        const int ld = rows + 1;
        const uint64_t other = right ? (uint64_t)cm * n : (uint64_t)m * cm;
        const uint64_t hw = (uint64_t)cm + ((uint64_t)cm * sizeof(int) + sizeof(V) - 1) / sizeof(V);
        const bool fast = (uint64_t)ld * cm + (uint64_t)cm * cm + other + hw <= P.x_smem;
        // the Gram-Schmidt matrix stays in shared memory whenever it fits there alone (R and the
        // projections then go to the slot's global scratch)
        const bool x_sh = (uint64_t)ld * cm <= P.x_smem;
        V* X = x_sh ? S.X : xg;
        V* Rm = fast || !x_sh ? X + (size_t)ld * cm : xg;  // R, row-major: kept index x cm
        V* O = fast ? Rm + (size_t)cm * cm : nullptr;       // staged copy of the other tensor
        V* hb = fast ? O + other : reinterpret_cast<V*>(gsig2);  // one pass's projections
        int* perm = reinterpret_cast<int*>(hb + cm);             // kept columns, in order
        V* A = site(q);
        V* B = site(q + 1);
        R fro = 0;
        if (right) {
#pragma unroll 1
            for (int e = tid_; e < m * cm; e += NT) {
                const int i = e / cm, j = e - i * cm;
                const V v = A[e];
                X[(size_t)j * ld + i] = v;
                fro = fma(v.x, v.x, fma(v.y, v.y, fro));
            }
            if (fast) for (int e = tid_; e < cm * n; e += NT) O[e] = B[e];
        } else {
#pragma unroll 1
            for (int e = tid_; e < cm * n; e += NT) {
                const int k = e / n, j = e - k * n;
                const V v = B[e];
                X[(size_t)k * ld + j] = cmk<V>(v.x, -v.y);
                fro = fma(v.x, v.x, fma(v.y, v.y, fro));
            }
            if (fast) for (int e = tid_; e < m * cm; e += NT) O[e] = A[e];
        }
#pragma unroll 1
        for (int e = tid_; e < cm * cm; e += NT) Rm[e] = cmk<V>(0, 0);
        const V* Bo = right ? (fast ? O : B) : B;
        const V* Ao = right ? A : (fast ? O : A);
        const double frod = (double)sum_r(fro);  // sets the numerical floor only: working precision
        const R eps = sizeof(R) == 4 ? (R)FLT_EPSILON : (R)DBL_EPSILON;
        const R fl = (R)4 * eps * sqrt((R)rows);
        const R floor2 = fl * fl * (R)frod;
        bsync<NT>();
        double dropped = 0;
        const int k = gram_schmidt(X, rows, cm, ld, Rm, hb, perm, floor2, dropped);
        const int r = k;
        if (r == 0) {  // a site tensor at the numerical floor: the state has lost its norm
            status = QC_ENOCONV;
            return;
        }
        if (dropped > 0 && frod > 0) disc += dropped / frod;
        if (right) {
            // A[q] = Q (cl, 2, r);  A[q+1] = R B (r, 2, cr), R upper triangular in column order
#pragma unroll 1
            for (int e = tid_; e < r * n; e += NT) {
                const int kk = e / n, jn = e - kk * n;
                const V* rrow = Rm + (size_t)kk * cm;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int j = perm[kk]; j < cm; ++j) acc = cfma(rrow[j], Bo[(size_t)j * n + jn], acc);
                tcopy[e] = acc;
            }
            bsync<NT>();
#pragma unroll 1
            for (int e = tid_; e < m * r; e += NT) {
                const int i = e / r, kk = e - i * r;
                A[e] = X[(size_t)kk * ld + i];
            }
#pragma unroll 1
            for (int e = tid_; e < r * n; e += NT) B[e] = tcopy[e];
        } else {
            // A[q+1] = Q^H (r, 2, cr);  A[q] = A[q] R^H (cl, 2, r)
#pragma unroll 1
            for (int e = tid_; e < m * r; e += NT) {
                const int i = e / r, kk = e - i * r;
                const V* rrow = Rm + (size_t)kk * cm;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int j = perm[kk]; j < cm; ++j) acc = cfmac(rrow[j], Ao[(size_t)i * cm + j], acc);
                tcopy[e] = acc;
            }
            bsync<NT>();
#pragma unroll 1
            for (int e = tid_; e < r * n; e += NT) {
                const int kk = e / n, jn = e - kk * n;
                const V u = X[(size_t)kk * ld + jn];
                B[e] = cmk<V>(u.x, -u.y);
            }
#pragma unroll 1
            for (int e = tid_; e < m * r; e += NT) A[e] = tcopy[e];
        }
        bsync<NT>();
        if (tid_ == 0) S.dims[q + 1] = r;
        bsync<NT>();
        tock(PH_MOVE);
        ++nupd;
        if (tid_ == 0) {  // Householder QR count of the rows x cm factor, plus the product with R
            const unsigned long long M = max(rows, cm), K = min(rows, cm);
            flops += (24ull * M * K * K - 8ull * K * K * K) / 3ull + 8ull * r * cm * (right ? n : m);
        }
    }

    // ---- SWAP with a qubit in a product state: a relabelling of bonds, no decomposition ---------
    // The unentangled qubit's tensor is |0> x M: its last readout left slice 1 at exactly zero, and
    // every single-qubit gate since then is still pending.  Product on the left (site q):
    // C = M A[q+1] (cl, 2, cr) goes to site q and |0> x I (cr, 2, cr) to site q+1.  Product on the
    // right: C = A[q] N (cl, 2, cr) goes to site q+1 and |0> x I (cl, 2, cl) to site q.  |0> x I is
    // an isometry either way, so the canonical form holds; a centre on the pair ends on the
    // entangled qubit's new site.  Pending gates travel with their qubits.
    // A readout can leave a bond wider than the state needs (the projection is not followed by a
    // split); when the new bond would exceed the rank bound of the other side (2 cl, resp. 2 cr) or
    // the bond capacity, C is factorised instead (LQ, resp. QR, by Gram-Schmidt) with the
    // orthonormal factor on the product qubit's new site, which keeps the canonical form.
    __device__ void pswap(int q, bool prod_left) {
        bsync<NT>();
        tick();
        const int cl = S.dims[q], cm = S.dims[q + 1], cr = S.dims[q + 2];
        V* A = site(q);
        V* B = site(q + 1);
        const int n = 2 * cr;
        R fro = 0;
        if (prod_left) {
#pragma unroll 1
            for (int e = tid_; e < cl * n; e += NT) {  // C(l, t, r) = sum_m A(l, 0, m) B(m, t, r)
                const int l = e / n, j = e - l * n;
                const V* arow = A + (size_t)(2 * l) * cm;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int k = 0; k < cm; ++k) acc = cfma(arow[k], B[(size_t)k * n + j], acc);
                tcopy[e] = acc;
                fro = fma(acc.x, acc.x, fma(acc.y, acc.y, fro));
            }
        } else {
#pragma unroll 1
            for (int e = tid_; e < 2 * cl * cr; e += NT) {  // C(l, s, r) = sum_m A(l, s, m) B(m, 0, r)
                const int i = e / cr, r = e - i * cr;
                const V* arow = A + (size_t)i * cm;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int k = 0; k < cm; ++k) acc = cfma(arow[k], B[(size_t)(2 * k) * cr + r], acc);
                tcopy[e] = acc;
                fro = fma(acc.x, acc.x, fma(acc.y, acc.y, fro));
            }
        }
        bsync<NT>();
        int nb = prod_left ? cr : cl;  // the new bond between q and q+1
        if (nb <= (prod_left ? 2 * cl : 2 * cr) && nb <= P.cap[q + 1]) {
            if (prod_left) {
#pragma unroll 1
                for (int e = tid_; e < cl * n; e += NT) A[e] = tcopy[e];
#pragma unroll 1
                for (int e = tid_; e < cr * n; e += NT) {
                    const int r1 = e / n, rem = e - r1 * n;
                    B[e] = cmk<V>(rem == r1 ? (R)1 : (R)0, (R)0);  // (r1, s = 0, r2 = r1)
                }
            } else {
#pragma unroll 1
                for (int e = tid_; e < 2 * cl * cr; e += NT) B[e] = tcopy[e];
#pragma unroll 1
                for (int e = tid_; e < cl * 2 * cl; e += NT) {
                    const int l1 = e / (2 * cl), rem = e - l1 * 2 * cl;
                    A[e] = cmk<V>(rem == l1 ? (R)1 : (R)0, (R)0);  // (l1, s = 0, l2 = l1)
                }
            }
        } else {
            // left: C as (2cl) x cr = L Q', by QR of C^H (cr x 2cl);  right: C as cl x (2cr) = Q R
            const int rows = prod_left ? cr : cl, cols = prod_left ? 2 * cl : 2 * cr;
            const int ld = rows + 1;
            const uint64_t hw = (uint64_t)cols + ((uint64_t)cols * sizeof(int) + sizeof(V) - 1) / sizeof(V);
            const uint64_t need = (uint64_t)ld * cols + (uint64_t)cols * cols;
            const bool fast = need + hw <= P.x_smem;
            const uint64_t sg_bytes = (uint64_t)(2 * P.chi_max) * (sizeof(R) + sizeof(int));
            if (!fast && (need > P.xg_elems || hw * sizeof(V) > sg_bytes)) {
                status = QC_ECAPACITY;
                return;
            }
            V* X = fast ? S.X : xg;
            V* Rm = X + (size_t)ld * cols;
            V* hb = fast ? Rm + (size_t)cols * cols : reinterpret_cast<V*>(gsig2);
            int* perm = reinterpret_cast<int*>(hb + cols);
#pragma unroll 1
            for (int e = tid_; e < rows * cols; e += NT) {
                if (prod_left) {  // X[r, j] = conj C[j, r]
                    const int j = e / cr, r = e - j * cr;
                    const V c = tcopy[e];
                    X[(size_t)j * ld + r] = cmk<V>(c.x, -c.y);
                } else {          // X[l, j] = C[l, j]
                    const int l = e / cols, j = e - l * cols;
                    X[(size_t)j * ld + l] = tcopy[e];
                }
            }
#pragma unroll 1
            for (int e = tid_; e < cols * cols; e += NT) Rm[e] = cmk<V>(0, 0);
            const double frod = (double)sum_r(fro);  // sets the numerical floor only: working precision
            const R eps = sizeof(R) == 4 ? (R)FLT_EPSILON : (R)DBL_EPSILON;
            const R fl = (R)4 * eps * sqrt((R)rows);
            const R floor2 = fl * fl * (R)frod;
            bsync<NT>();
            double dropped = 0;
            const int k = gram_schmidt(X, rows, cols, ld, Rm, hb, perm, floor2, dropped);
            if (k == 0) {
                status = QC_ENOCONV;
                return;
            }
            if (k > P.cap[q + 1]) {
                status = QC_ECAPACITY;
                return;
            }
            if (dropped > 0 && frod > 0) disc += dropped / frod;
            nb = k;
            if (prod_left) {
                // A[q](l, t, kk) = conj R[kk, (l, t)];  A[q+1](kk, s, r) = [s = 0] conj Q[r, kk]
#pragma unroll 1
                for (int e = tid_; e < cols * k; e += NT) {
                    const int j = e / k, kk = e - j * k;
                    const V u = Rm[(size_t)kk * cols + j];
                    A[e] = cmk<V>(u.x, -u.y);
                }
#pragma unroll 1
                for (int e = tid_; e < k * n; e += NT) {
                    const int kk = e / n, rem = e - kk * n;
                    V v = cmk<V>(0, 0);
                    if (rem < cr) {
                        const V u = X[(size_t)kk * ld + rem];
                        v = cmk<V>(u.x, -u.y);
                    }
                    B[e] = v;
                }
            } else {
                // A[q](l, t, kk) = [t = 0] Q[l, kk];  A[q+1](kk, s, r) = R[kk, (s, r)]
#pragma unroll 1
                for (int e = tid_; e < cl * 2 * k; e += NT) {
                    const int l = e / (2 * k), rem = e - l * 2 * k;
                    A[e] = rem < k ? X[(size_t)rem * ld + l] : cmk<V>(0, 0);
                }
#pragma unroll 1
                for (int e = tid_; e < k * cols; e += NT) B[e] = Rm[e];
            }
            if (tid_ == 0) {
                const unsigned long long M = max(rows, cols), K = min(rows, cols);
                flops += (24ull * M * K * K - 8ull * K * K * K) / 3ull;
            }
        }
        bsync<NT>();
        if (tid_ == 0) {
            S.dims[q + 1] = nb;
#pragma unroll 1
            for (int k = 0; k < 4; ++k) {
                const V t = S.pend[q * 4 + k];
                S.pend[q * 4 + k] = S.pend[(q + 1) * 4 + k];
                S.pend[(q + 1) * 4 + k] = t;
            }
            flops += 16ull * cl * cm * cr;
        }
        bsync<NT>();
        tock(PH_PSWAP);
        chi_peak = max(chi_peak, nb);
    }

    // ---- readout on site q (the orthogonality centre) ------------------------------------------
    // returns the outcome, or -1 when the shot ends (rejected / error)
    __device__ int readout(int q, uint32_t rid, bool is_meas, uint64_t shot, int64_t src) {
        bsync<NT>();  // pending gates written by thread 0
        tick();
        const int cl = S.dims[q], cr = S.dims[q + 1];
        V* a = site(q);
        const V* u = S.pend + q * 4;
        const V g00 = u[0], g01 = u[1], g10 = u[2], g11 = u[3];
        double p0 = 0, p1 = 0;
#pragma unroll 1
        for (int e = tid_; e < cl * cr; e += NT) {
            const int l = e / cr, r = e - l * cr;
            V* px = a + (l * 2) * cr + r;
            V* py = px + cr;
            const V x0 = *px, y0 = *py;
            const V x = cfma(g00, x0, cmul(g01, y0)), y = cfma(g10, x0, cmul(g11, y0));
            *px = x;
            *py = y;
            p0 += (double)x.x * x.x + (double)x.y * x.y;
            p1 += (double)y.x * y.x + (double)y.y * y.y;
        }
        p0 = block_sum<NT>(p0, S.red, tid_);
        p1 = block_sum<NT>(p1, S.red, tid_);
        if (tid_ == 0) reset_pend(q);
        const double tot = p0 + p1;
        const double pr1 = tot > 0 ? p1 / tot : 0.0;
        if (P.trace_p1 && !P.reference && rid < (uint32_t)P.trace_k && tid_ == 0) {
            const uint64_t row = P.trace_pos ? P.trace_pos[task_] : task_;
            P.trace_p1[row * (uint64_t)P.trace_k + rid] = pr1;
        }
        int outcome;
        if (P.reference) {
            if (is_meas) {
                const double lim = P.precision == QC_C128 ? 1e-10 : 1e-5;
                if (pr1 > lim) {
                    if (tid_ == 0) atomicCAS(P.ref_status, 0, (int)(src + 1));
                }
                outcome = 0;
            } else {
                // a reset of an undetermined qubit: fixed convention, robust to rounding at p1 = 1/2
                outcome = pr1 > 0.6180339887498949 ? 1 : 0;
            }
        } else {
            const double u = readout_uniform(rid, shot, P.k0, P.k1);
            outcome = u < pr1 ? 1 : 0;
        }
        if (is_meas && outcome == 1) {
            status = 1;
            abort_op = src;
            return -1;
        }
        const double po = outcome ? p1 : p0;
        if (!(po > 0)) {  // projection onto a zero-probability branch cannot happen for draws
            status = QC_EINVAL;
            return -1;
        }
        const R sc = (R)(1.0 / sqrt(po));
        const bool flip = (!is_meas) && outcome == 1;  // reset to |0>: project on 1 then X
#pragma unroll 1
        for (int e = tid_; e < cl * cr; e += NT) {
            const int l = e / cr, r = e - l * cr;
            V* x0 = a + (l * 2) * cr + r;
            V* x1 = x0 + cr;
            const V keep = outcome ? *x1 : *x0;
            const V kv = cmk<V>(keep.x * sc, keep.y * sc);
            if (outcome == 0) { *x0 = kv; *x1 = cmk<V>(0, 0); }
            else if (flip) { *x0 = kv; *x1 = cmk<V>(0, 0); }
            else { *x0 = cmk<V>(0, 0); *x1 = kv; }
        }
        bsync<NT>();
        tock(PH_READOUT);
        return outcome;
    }

    // ---- <ref|psi> by a transfer sweep ----------------------------------------------------------
    __device__ double2 overlap_ref() {
        // E: (chi_ref x chi), T1: (chi_ref x 2 x chi); placed in shared X when it fits
        const int cap2 = max(P.chi_max, P.ref_chi);  // bounds the bonds of both states
        const uint64_t need = (uint64_t)cap2 * cap2 * 3;
        V* E = (need <= P.x_smem) ? S.X : xg;
        V* T1 = E + (size_t)cap2 * cap2;
        if (tid_ == 0) E[0] = cmk<V>(1, 0);
        bsync<NT>();
        const V* refsite = P.ref;
#pragma unroll 1
        for (int q = 0; q < P.nq; ++q) {
            const int ca = P.ref_dims[q], ca2 = P.ref_dims[q + 1];
            const int cb = S.dims[q], cb2 = S.dims[q + 1];
            const V* Aq = site(q);
            const V* Rq = refsite + P.ref_off[q];
            // T1[a][s][b'] = sum_b E[a][b] A[b][s][b']
#pragma unroll 1
            for (int e = tid_; e < ca * 2 * cb2; e += NT) {
                const int a_ = e / (2 * cb2), rest = e - a_ * 2 * cb2;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int b = 0; b < cb; ++b) acc = cfma(E[(size_t)a_ * cb + b], Aq[(size_t)b * 2 * cb2 + rest], acc);
                T1[e] = acc;
            }
            bsync<NT>();
            // E'[a'][b'] = sum_{a,s} conj(R[a][s][a']) T1[a][s][b']
#pragma unroll 1
            for (int e = tid_; e < ca2 * cb2; e += NT) {
                const int ap = e / cb2, bp = e - ap * cb2;
                V acc = cmk<V>(0, 0);
#pragma unroll 1
                for (int a_ = 0; a_ < ca; ++a_)
#pragma unroll 1
                    for (int s = 0; s < 2; ++s)
                        acc = cfmac(Rq[((size_t)a_ * 2 + s) * ca2 + ap], T1[((size_t)a_ * 2 + s) * cb2 + bp], acc);
                E[e] = acc;
            }
            bsync<NT>();
        }
        const V ov = E[0];
        bsync<NT>();
        return make_double2((double)ov.x, (double)ov.y);
    }

    __device__ double centre_norm2(const V* base, const int* dims) {
        const int q = P.final_center;
        const int cl = dims[q], cr = dims[q + 1];
        const V* a = base + P.off[q];
        double s = 0;
#pragma unroll 1
        for (int e = tid_; e < cl * 2 * cr; e += NT) s += (double)a[e].x * a[e].x + (double)a[e].y * a[e].y;
        return block_sum<NT>(s, S.red, tid_);
    }

    // ---- faults of one shot into S.fch / S.fcode (sorted by channel); returns the count ------
    __device__ int faults(uint64_t shot) {
        int& nf = *S.nf;
        if (tid_ == 0) nf = 0;
        bsync<NT>();
        if (P.reference) return 0;
        if (P.weight < 0) {
            const uint32_t w = (uint32_t)(shot >> 6), lane = (uint32_t)(shot & 63);
            const uint32_t ng = (P.nchan + 3) / 4;
#pragma unroll 1
            for (uint32_t g = tid_; g < ng; g += NT) {
                const U4 u = philox(g, w, 0, TAG_WORD, P.k0, P.k1);
#pragma unroll
                for (uint32_t j = 0; j < 4; ++j) {
                    const uint32_t c = g * 4 + j;
                    const uint32_t u0 = u4_get(u, j);
                    if (c >= P.nchan || u0 >= P.tg[63]) continue;
                    const uint64_t msk = lane_mask(u0, c, w, P.tg, P.k0, P.k1);
                    if (!((msk >> lane) & 1)) continue;
                    const int slot_i = atomicAdd(&nf, 1);
                    if (slot_i < MAXF) {
                        S.fch[slot_i] = c;
                        S.fcode[slot_i] = (uint8_t)fault_code(P.chan_kind[c], c, w, lane, P.k0, P.k1);
                    }
                }
            }
            bsync<NT>();
            if (tid_ == 0) {  // insertion sort by channel
                const int cnt = min(nf, MAXF);
#pragma unroll 1
                for (int i = 1; i < cnt; ++i) {
                    const uint32_t c = S.fch[i];
                    const uint8_t d = S.fcode[i];
                    int k = i;
                    while (k > 0 && S.fch[k - 1] > c) { S.fch[k] = S.fch[k - 1]; S.fcode[k] = S.fcode[k - 1]; --k; }
                    S.fch[k] = c;
                    S.fcode[k] = d;
                }
            }
        } else if (tid_ == 0) {
            uint32_t draw = 0;
            const uint32_t M = P.nchan, W = (uint32_t)P.weight;
            int cnt = 0;
#pragma unroll 1
            for (uint32_t j = M - W; j < M; ++j) {
                const uint32_t t = exact_bounded(shot, draw, j + 1, P.k0, P.k1);
                bool present = false;
#pragma unroll 1
                for (int k = 0; k < cnt; ++k) present |= (S.fch[k] == t);
                const uint32_t v = present ? j : t;
                if (cnt < MAXF) {
                    int k = cnt;
                    while (k > 0 && S.fch[k - 1] > v) { S.fch[k] = S.fch[k - 1]; --k; }
                    S.fch[k] = v;
                }
                ++cnt;
            }
#pragma unroll 1
            for (int k = 0; k < min(cnt, MAXF); ++k) S.fcode[k] = (uint8_t)exact_code(P.chan_kind[S.fch[k]], S.fch[k], shot, P.k0, P.k1);
            nf = cnt;
        }
        bsync<NT>();
        const int out = nf;
        bsync<NT>();
        return out;
    }

    __device__ void run(uint64_t task) {
        task_ = task;
        const uint64_t shot = P.reference ? 0 : P.shots[task];
        status = 0; disc = 0; degen = 0; chi_peak = 1; nupd = 0; abort_op = -1; flops = 0; sweeps = 0;
        gmem_updates = 0;
        resplits = 0;
#pragma unroll 1
        for (int q = tid_; q <= P.nq; q += NT) S.dims[q] = 1;
#pragma unroll 1
        for (int q = tid_; q < P.nq; q += NT) {
            V* a = site(q);
            a[0] = cmk<V>(1, 0);
            a[1] = cmk<V>(0, 0);
            reset_pend(q);
        }
        if (P.phase_cycles && tid_ == 0)
#pragma unroll 1
            for (int k = 0; k < 8; ++k) S.phase[k] = 0;
        bsync<NT>();
        tick();
        const int nf = faults(shot);
        tock(PH_FAULTS);
        if (nf > MAXF) status = QC_ECAPACITY;
#pragma unroll 1
        for (uint32_t base = 0; base < P.nops && status == 0; base += OPCH) {
            const uint32_t cnt = min((uint32_t)OPCH, P.nops - base);
#pragma unroll 1
            for (uint32_t i = tid_; i < cnt; i += NT) S.ops[i] = P.prog[base + i];
            bsync<NT>();
#pragma unroll 1
            for (uint32_t i = 0; i < cnt && status == 0; ++i) {
                const MpsOp op = S.ops[i];
                switch (op.kind) {
                    case M_G1: {
                        const V* g = P.g1 + op.a * 4;
                        defer1(op.q, g[0], g[1], g[2], g[3]);
                        break;
                    }
                    case M_CH1:
                    case M_CH2: {
                        // the schedule may visit channels out of text order: binary search the
                        // shot's faults (sorted by channel)
                        int lo = 0, hi = nf;
                        while (lo < hi) {
                            const int mid = (lo + hi) >> 1;
                            if (S.fch[mid] < op.a) lo = mid + 1; else hi = mid;
                        }
                        if (lo < nf && S.fch[lo] == op.a) {
                            const uint32_t code = S.fcode[lo];
                            if (op.kind == M_CH1) defer_pauli(op.q, code);
                            else { defer_pauli(op.q, code >> 2); defer_pauli(op.b, code & 3); }
                        }
                        break;
                    }
                    case M_G2:
                        update(op.q, P.g4 + op.a * 16, (op.flags & F_CENTER_RIGHT) != 0);
                        if (status != 0) abort_op = op.src;
                        break;
                    case M_MOVE:
                        move(op.q, (op.flags & F_CENTER_RIGHT) != 0);
                        break;
                    case M_PSWAP:
                        pswap(op.q, (op.flags & F_PROD_LEFT) != 0);
                        break;
                    case M_MEAS:
                    case M_RESET:
                        readout(op.q, op.a, op.kind == M_MEAS, shot, op.src);
                        break;
                    default: break;
                }
            }
            bsync<NT>();
        }
        // finish: apply the gates still pending, then compare with the reference
        tick();
        if (status == 0)
#pragma unroll 1
            for (int q = 0; q < P.nq; ++q) {
                bsync<NT>();
                const V* u = S.pend + q * 4;
                const bool ident = u[0].x == (R)1 && u[0].y == (R)0 && u[1].x == (R)0 && u[1].y == (R)0 &&
                                   u[2].x == (R)0 && u[2].y == (R)0 && u[3].x == (R)1 && u[3].y == (R)0;
                if (!ident) flush_site(q);
            }
        bsync<NT>();
        double fid = -1.0;
        int lerr = 0;
        if (status == 0 && !P.reference) {
            const double2 ov = overlap_ref();
            const double nn = centre_norm2(slot, S.dims);
            const double ov2 = ov.x * ov.x + ov.y * ov.y;
            fid = (nn > 0 && P.ref_norm > 0) ? ov2 / (nn * P.ref_norm) : 0.0;
            double tau = P.tau;
            if (!(tau > 0)) tau = P.precision == QC_C128 ? 1e-8 : fmax(1e-3, 10.0 * (P.ref_disc + disc));
            lerr = (1.0 - fid) > tau;
        }
        if (tid_ == 0) {
            if (P.reference) {
#pragma unroll 1
                for (int q = 0; q <= P.nq; ++q) P.ref_dims_out[q] = S.dims[q];
                *P.ref_disc_out = disc;
                *P.ref_chi_out = chi_peak;
                if (status != 0) atomicCAS(P.ref_status, 0, -1000 + status);
            } else if (!(P.defer_capacity && (status == QC_ECAPACITY || status == QC_INTERNAL_FP64_RERUN))) {
                const int wb = min(nf, P.wmax);
                atomicAdd(&P.counts[3 * wb + 0], 1ull);
                if (status == 0) {
                    atomicAdd(&P.counts[3 * wb + 1], 1ull);
                    if (lerr) atomicAdd(&P.counts[3 * wb + 2], 1ull);
                }
            }
            if (!P.reference) {
                if (P.per_shot) {
                    qc_shot_result res;
                    res.shot = shot;
                    res.status = status;
                    res.weight = nf;
                    res.logical_error = lerr;
                    res.chi_peak = chi_peak;
                    res.abort_op = abort_op;
                    res.fidelity = fid;
                    res.discarded = disc;
                    res.degenerate_cuts = degen;
                    res.n_updates = nupd;
                    res.alg_flops = (double)flops;
                    res.sweeps = sweeps;
                    res.gmem_updates = gmem_updates;
                    res.fp64_resplits = resplits;
                    P.per_shot[task] = res;
                }
            }
        }
        tock(PH_FINISH);
        if (P.phase_cycles && tid_ == 0 && !P.reference)
#pragma unroll 1
            for (int k = 0; k < 8; ++k) atomicAdd(&P.phase_cycles[k], S.phase[k]);
        bsync<NT>();
    }
};

template <typename R, int NT>
__host__ __device__ size_t engine_smem(const EngineParams<R>& P);

// Shared-memory layout of one engine's region (X, program chunk, reductions, bonds, pending gates,
// fused gate, faults).
template <typename R>
__device__ unsigned char* carve(Shared<R>& S, unsigned char* p, const EngineParams<R>& P) {
    using V = typename VecOf<R>::T;
    S.X = reinterpret_cast<V*>(p); p += (size_t)P.x_smem * sizeof(V);
    S.ops = reinterpret_cast<MpsOp*>(p); p += OPCH * sizeof(MpsOp);
    S.red = reinterpret_cast<double*>(p); p += 64 * sizeof(double);
    S.dims = reinterpret_cast<int*>(p); p += (size_t)(P.nq + 1) * sizeof(int);
    p = reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
    S.pend = reinterpret_cast<V*>(p); p += (size_t)P.nq * 4 * sizeof(V);
    S.gate = reinterpret_cast<V*>(p); p += 16 * sizeof(V);
    S.fch = reinterpret_cast<uint32_t*>(p); p += MAXF * sizeof(uint32_t);
    S.nf = reinterpret_cast<int*>(p); p += 16;
    S.phase = reinterpret_cast<unsigned long long*>(p); p += 8 * sizeof(unsigned long long);
    S.t_mark = reinterpret_cast<long long*>(p); p += 16;
    S.mbar = reinterpret_cast<uint64_t*>(p); p += 8;
    S.tmem_slot = reinterpret_cast<uint32_t*>(p); p += 8;
    S.fcode = reinterpret_cast<uint8_t*>(p); p += MAXF;
    return reinterpret_cast<unsigned char*>(((uintptr_t)p + 15) & ~(uintptr_t)15);
}

// Persistent engine.  CTA mode (NT > 32): the CTA is one engine.  Warp mode (NT = 32): every warp
// of the CTA is an engine with its own shot slot, and the warps share one large work area.
template <typename R, int NT>
__global__ void __launch_bounds__(NT == 32 ? 256 : NT, NT == 32 ? 2 : (NT == 128 ? 4 : (NT == 256 ? 2 : 1)))
engine_kernel(const EngineParams<R> P) {
    unsigned char* smem_raw = qc_dsmem;
    const int engines = (NT == 32) ? (int)(blockDim.x >> 5) : 1;
    const int e = (NT == 32) ? (int)(threadIdx.x >> 5) : 0;
    const int tid = (NT == 32) ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
    const size_t region = (engine_smem<R, NT>(P) + 15) & ~(size_t)15;
    Shared<R> S;
    carve<R>(S, smem_raw + region * e, P);
    S.big = reinterpret_cast<typename VecOf<R>::T*>(smem_raw + region * engines);
    S.big_lock = reinterpret_cast<int*>(smem_raw + region * engines + (size_t)P.x_big * sizeof(typename VecOf<R>::T));
    if (NT == 32 && threadIdx.x == 0) *S.big_lock = 0;
    __syncthreads();
    Engine<R, NT> eng(P, S, blockIdx.x * engines + e, tid);
    if constexpr (NT >= 128) {
        if (P.use_tc) {  // 128 tensor-memory columns per CTA (the host admits at most 4 CTAs per SM)
            if (threadIdx.x < 32) qc::tc::tmem_alloc(S.tmem_slot, 128);
            if (threadIdx.x == 0) qc::tc::mbar_init(S.mbar, 1);
            qc::tc::fence_before_sync();
            __syncthreads();
            qc::tc::fence_after_sync();
            eng.tmem_ = *S.tmem_slot;
        }
    }
    for (;;) {
        unsigned long long task = 0;
        if (NT == 32) {
            if (tid == 0) task = atomicAdd(P.next_task, 1ull);
            task = __shfl_sync(0xFFFFFFFFu, task, 0);
        } else {
            __shared__ unsigned long long task_s;
            if (tid == 0) task_s = atomicAdd(P.next_task, 1ull);
            __syncthreads();
            task = task_s;
            __syncthreads();
        }
        if (task >= P.ntasks) break;
        eng.run(task);
    }
    if constexpr (NT >= 128) {
        if (P.use_tc) {
            qc::tc::fence_before_sync();
            __syncthreads();
            qc::tc::fence_after_sync();
            if (threadIdx.x < 32) qc::tc::tmem_dealloc(eng.tmem_, 128);
        }
    }
}

// Bytes of one engine's region.
template <typename R, int NT>
__host__ __device__ size_t engine_smem(const EngineParams<R>& P) {
    using V = typename VecOf<R>::T;
    return (size_t)P.x_smem * sizeof(V) + OPCH * sizeof(MpsOp) + 64 * sizeof(double) +
           (size_t)(P.nq + 1) * sizeof(int) + 16 + (size_t)P.nq * 4 * sizeof(V) + 16 * sizeof(V) +
           MAXF * sizeof(uint32_t) + 16 + 8 * sizeof(unsigned long long) + 16 + 16 + MAXF + 16;
}

// ---- gate tables ------------------------------------------------------------------------------
void gate_tables(std::vector<double2>& g1, std::vector<double2>& g4) {
    const double h = std::sqrt(0.5), c8 = std::cos(M_PI / 4), s8 = std::sin(M_PI / 4);
    g1.assign(G1_COUNT * 4, make_double2(0, 0));
    auto set1 = [&](int gi, double2 a, double2 b, double2 c, double2 d) {
        g1[gi * 4 + 0] = a; g1[gi * 4 + 1] = b; g1[gi * 4 + 2] = c; g1[gi * 4 + 3] = d;
    };
    const double2 z = make_double2(0, 0), o = make_double2(1, 0);
    set1(G1_H, make_double2(h, 0), make_double2(h, 0), make_double2(h, 0), make_double2(-h, 0));
    set1(G1_S, o, z, z, make_double2(0, 1));
    set1(G1_SDG, o, z, z, make_double2(0, -1));
    set1(G1_X, z, o, o, z);
    set1(G1_Y, z, make_double2(0, -1), make_double2(0, 1), z);
    set1(G1_Z, o, z, z, make_double2(-1, 0));
    set1(G1_T, o, z, z, make_double2(c8, s8));
    set1(G1_TDG, o, z, z, make_double2(c8, -s8));
    g4.assign(G4_COUNT * 16, z);
    auto set4 = [&](int gi, int row, int col, double2 v) { g4[gi * 16 + row * 4 + col] = v; };
    // index (s,t) = 2*s + t with s the site q (high bit)
    // CX control high, target low: |s t> -> |s, t^s>
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) set4(G4_CX_HL, 2 * s + (t ^ s), 2 * s + t, o);
    // CX control low, target high
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) set4(G4_CX_LH, 2 * (s ^ t) + t, 2 * s + t, o);
    for (int k = 0; k < 4; ++k) set4(G4_CZ, k, k, k == 3 ? make_double2(-1, 0) : o);
    for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) set4(G4_SWAP, 2 * t + s, 2 * s + t, o);
    for (int k = 0; k < 4; ++k) set4(G4_ID, k, k, o);
}

struct DeviceTables {
    double2* g1d = nullptr;
    double2* g4d = nullptr;
    float2* g1f = nullptr;
    float2* g4f = nullptr;
};

std::mutex g_tab_mu;
std::map<int, DeviceTables> g_tables;

qc_status device_tables(DeviceTables** out) {
    int d = 0;
    QC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(g_tab_mu);
    auto it = g_tables.find(d);
    if (it == g_tables.end()) {
        std::vector<double2> g1, g4;
        gate_tables(g1, g4);
        std::vector<float2> f1(g1.size()), f4(g4.size());
        for (size_t i = 0; i < g1.size(); ++i) f1[i] = make_float2((float)g1[i].x, (float)g1[i].y);
        for (size_t i = 0; i < g4.size(); ++i) f4[i] = make_float2((float)g4[i].x, (float)g4[i].y);
        DeviceTables t;
        QC_CUDA(cudaMalloc(&t.g1d, g1.size() * sizeof(double2)));
        QC_CUDA(cudaMalloc(&t.g4d, g4.size() * sizeof(double2)));
        QC_CUDA(cudaMalloc(&t.g1f, f1.size() * sizeof(float2)));
        QC_CUDA(cudaMalloc(&t.g4f, f4.size() * sizeof(float2)));
        QC_CUDA(cudaMemcpy(t.g1d, g1.data(), g1.size() * sizeof(double2), cudaMemcpyHostToDevice));
        QC_CUDA(cudaMemcpy(t.g4d, g4.data(), g4.size() * sizeof(double2), cudaMemcpyHostToDevice));
        QC_CUDA(cudaMemcpy(t.g1f, f1.data(), f1.size() * sizeof(float2), cudaMemcpyHostToDevice));
        QC_CUDA(cudaMemcpy(t.g4f, f4.data(), f4.size() * sizeof(float2), cudaMemcpyHostToDevice));
        it = g_tables.emplace(d, t).first;
    }
    *out = &it->second;
    return QC_OK;
}

constexpr int NT_F = 512;
constexpr int NT_D = 256;

}  // namespace

// Layout of one slot: bond capacities and site offsets.
struct SlotLayout {
    std::vector<int> cap;
    std::vector<uint64_t> off;
    int chi_cap;
    uint64_t stride;
};

static SlotLayout slot_layout(int n, int chi_max) {
    SlotLayout L;
    L.cap.assign(n + 1, 1);
    L.chi_cap = 1;
    for (int k = 1; k < n; ++k) {
        const int e = std::min(k, n - k);
        const int64_t full = e >= 30 ? (int64_t)1 << 30 : (int64_t)1 << e;
        L.cap[k] = (int)std::min<int64_t>(full, chi_max);
        L.chi_cap = std::max(L.chi_cap, L.cap[k]);
    }
    L.off.assign(n + 1, 0);
    for (int q = 0; q < n; ++q) L.off[q + 1] = L.off[q] + (uint64_t)L.cap[q] * 2 * L.cap[q + 1];
    L.stride = (L.off[n] + 1) & ~1ull;
    return L;
}

// Elements of one slot's split scratch for slots of capacity chi next to a reference state whose largest
// bond is ref_chi: the Jacobi / overlap work area X, the theta' copy, and the singular values with their
// order.  Used for the allocation and for the admission footprint, so both always agree.
static uint64_t scratch_elems(int chi, int ref_chi, size_t sizeR, size_t sizeV) {
    const uint64_t cap2 = (uint64_t)std::max(chi, ref_chi);
    const uint64_t x_full = (uint64_t)(2 * chi + 1) * (2 * chi);
    const uint64_t xg_elems = std::max(x_full, cap2 * cap2 * 3);
    const uint64_t sg_elems = ((uint64_t)(2 * chi) * (sizeR + sizeof(int)) + sizeV - 1) / sizeV + 2;
    const uint64_t base = xg_elems + (uint64_t)(2 * chi) * (2 * chi) + sg_elems;
    if (sizeR == 4) {  // complex64: room for an FP64 re-split (X, theta' and the spectrum in double)
        const uint64_t c2 = (uint64_t)(2 * chi);
        const uint64_t fp64 = 2 * ((c2 + 1) * c2 + c2 * c2) + (c2 * (sizeof(double) + sizeof(int)) + sizeV - 1) / sizeV + 2;
        return std::max(base, fp64);
    }
    return base;
}

// Capacity bucket of the first pass: 64 when the reference's chi_peak is at most 64 (the warp variant's
// design size: theta at most 128 x 128; shots that outgrow it go to the re-run pass, which runs one CTA
// per shot), otherwise the smallest power of two >= 2 x the reference's chi_peak; at most the full
// capacity chi (QCMPS_CHI_ALLOC overrides it for tests and tuning).
static int bucket_chi(int ref_chi_peak, int chi) {
    int chi_alloc = 64;
    while (ref_chi_peak > 64 && chi_alloc < 2 * ref_chi_peak) chi_alloc *= 2;
    chi_alloc = std::min(chi_alloc, chi);
    if (const char* ca = getenv("QCMPS_CHI_ALLOC")) chi_alloc = std::max(1, std::min(chi, atoi(ca)));
    return chi_alloc;
}

// Shared-memory configuration of one engine variant: how much of theta's Jacobi matrix X fits in
// shared memory next to the fixed per-CTA arrays, within the variant's budget.
template <typename R, int NT>
static size_t configure_smem(EngineParams<R>& P, size_t budget, uint64_t x_full) {
    using V = typename VecOf<R>::T;
    P.x_smem = 0;
    const uint64_t fixed = engine_smem<R, NT>(P);
    uint64_t x_cap = (budget - std::min<uint64_t>(budget, fixed)) / sizeof(V);
    P.x_smem = (uint32_t)(std::min<uint64_t>(x_cap, x_full) & ~1ull);  // keeps the next region 16-byte aligned
    return engine_smem<R, NT>(P);
}

// Launch configuration of the persistent engine: threads per shot (32 = one warp per shot, several
// shot slots per SM; 128 / 256 / 512 = one CTA per shot) and the shared-memory work area per engine.
struct LaunchCfg {
    int variant;  // 32, 128, 256 or 512 (the large CTA)
    int kb;       // work area per engine, KB
    int warps;    // warp variant: engines per CTA sharing a large area (1 = none)
    int big_kb;   // warp variant: the shared large area, KB
};

// One persistent launch over `nshots` shots with slots of layout L (reference stored in L).
template <typename R, int NT_BIG>
static qc_status run_pass(CircuitImpl& c, EngineParams<R> P, const SlotLayout& L, const void* ref_state,
                          const int* cap_dev, const uint64_t* off_dev, const RefState& ref,
                          const uint64_t* shots_dev, uint64_t nshots, unsigned long long* counts_dev,
                          qc_shot_result* per_shot, cudaStream_t s, int max_slots, int nsm, bool defer,
                          LaunchCfg cfg) {
    using V = typename VecOf<R>::T;
    const int chi = P.chi_max;
    P.ref_chi = std::max(1, ref.chi_peak);
    const uint64_t cap2 = (uint64_t)std::max(chi, P.ref_chi);
    const uint64_t x_full = (uint64_t)(2 * chi + 1) * (2 * chi);
    const uint64_t over_full = cap2 * cap2 * 3;
    const uint64_t xg_elems = std::max(x_full, over_full);
    const uint64_t scratch_stride = scratch_elems(chi, P.ref_chi, sizeof(R), sizeof(V));
    P.slot_stride = L.stride;
    P.scratch_stride = scratch_stride;
    P.xg_elems = xg_elems;
    P.defer_capacity = defer ? 1 : 0;
    const int variant = cfg.variant;
    const int kbv = cfg.kb;
    size_t smem;
    int nt = variant;
    int engines = 1;  // engines (shot slots) per CTA
    const void* fn;
    if (variant == 32) {
        // measured on the 49-qubit workload: one warp per CTA with 24 KB (9 shot slots per SM)
        // beats sharing a large area between warps (contention) and larger per-warp areas (fewer
        // slots)
        engines = (cfg.warps >= 1 && cfg.warps <= 8) ? cfg.warps : 1;
        const size_t per = configure_smem<R, 32>(P, (kbv >= 8 && kbv <= 200 ? kbv : 24) * 1024, xg_elems);
        const size_t region = (per + 15) & ~(size_t)15;
        const size_t big_budget = cfg.big_kb > 0 ? (size_t)cfg.big_kb * 1024 : 0;
        size_t room = 227 * 1024 > region * engines + 16 ? 227 * 1024 - region * engines - 16 : 0;
        if (engines == 1) room = 0;  // nobody to share with
        room = std::min(room, big_budget);
        P.x_big = (uint32_t)std::min<uint64_t>((room / sizeof(V)) & ~1ull, 4 * xg_elems);
        smem = region * engines + (size_t)P.x_big * sizeof(V) + 16;
        fn = (const void*)engine_kernel<R, 32>;
        nt = 32 * engines;
    } else if (variant == 128) {
        smem = configure_smem<R, 128>(P, (kbv >= 8 && kbv <= 200 ? kbv : 72) * 1024, xg_elems);
        fn = (const void*)engine_kernel<R, 128>;
    } else if (variant == 256) {
        smem = configure_smem<R, 256>(P, (kbv >= 8 && kbv <= 200 ? kbv : 100) * 1024, xg_elems);
        fn = (const void*)engine_kernel<R, 256>;
    } else {
        smem = configure_smem<R, NT_BIG>(P, (kbv >= 8 && kbv <= 220 ? kbv : 200) * 1024, xg_elems);
        fn = (const void*)engine_kernel<R, NT_BIG>;
        nt = NT_BIG;
    }
    {
        const qc_status so = smem_optin(fn);
        if (so != QC_OK) return so;
    }
    int per_sm = 0;
    QC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
    if (per_sm < 1) return fail(QC_ENOMEM, "engine does not fit on an SM (smem %zu)", smem);
    // tensor-core contractions: complex64 CTA variants only, and only while every CTA that can be
    // resident on an SM gets its 128 tensor-memory columns (512 per SM) without waiting
    {
        const char* tcv = getenv("QCMPS_TC");
        P.use_tc = (sizeof(R) == 4 && variant >= 128 && per_sm * 128 <= 512 && !(tcv && atoi(tcv) == 0)) ? 1 : 0;
    }
    uint64_t ctas = std::min<uint64_t>((nshots + engines - 1) / engines, (uint64_t)per_sm * nsm);
    if (max_slots > 0) ctas = std::min<uint64_t>(ctas, std::max<uint64_t>(1, (uint64_t)max_slots / engines));
    if (ctas < 1) ctas = 1;
    const uint64_t slots = ctas * engines;

    const uint64_t mps_elems = slots * L.stride;
    const uint64_t scr_elems = slots * scratch_stride;
    char* ws = nullptr;
    const size_t bytes = (mps_elems + scr_elems) * sizeof(V) + 64;
    cudaError_t e = cudaMallocAsync((void**)&ws, bytes, s);
    if (e != cudaSuccess) return fail(QC_ENOMEM, "workspace of %zu bytes: %s", bytes, cudaGetErrorString(e));
    qc_status out = QC_OK;
    do {
        V* mps = reinterpret_cast<V*>(ws + 64);
        V* scr = mps + mps_elems;
        e = cudaMemsetAsync(ws, 0, 64, s);
        if (e != cudaSuccess) { out = cuda_fail(e, "workspace init"); break; }
        P.reference = 0;
        P.mps = mps;
        P.off = off_dev;
        P.cap = cap_dev;
        P.scratch = scr;
        P.ref = reinterpret_cast<const V*>(ref_state);
        P.ref_off = ref.off;
        P.ref_dims = ref.dims;
        P.ref_disc = ref.disc;
        P.ref_norm = ref.norm;
        P.shots = shots_dev;
        P.ntasks = nshots;
        P.next_task = reinterpret_cast<unsigned long long*>(ws);
        P.per_shot = per_shot;
        P.counts = counts_dev;
        if (variant == 32) engine_kernel<R, 32><<<(unsigned)ctas, 32 * engines, smem, s>>>(P);
        else if (variant == 128) engine_kernel<R, 128><<<(unsigned)ctas, 128, smem, s>>>(P);
        else if (variant == 256) engine_kernel<R, 256><<<(unsigned)ctas, 256, smem, s>>>(P);
        else engine_kernel<R, NT_BIG><<<(unsigned)ctas, NT_BIG, smem, s>>>(P);
        e = cudaGetLastError();
        if (e != cudaSuccess) { out = cuda_fail(e, "engine"); break; }
    } while (0);
    cudaFreeAsync(ws, s);
    return out;
}

// The launch rule without measurement: one warp per shot (24 KB work area) for small passes (the first
// pass of a circuit whose noiseless run stays at bond 64) when the batch fills the SMs or shares the GPU
// with other batches; otherwise one CTA per shot -- 128 threads with 72 KB when sharing the GPU (it finds
// room beside other batches' warps), else 512 threads with 200 KB (the lowest latency per shot).  The
// re-run pass of shots that outgrew the capacity bucket always takes the 512-thread CTA: its shots have
// large theta, and in smaller engines they would hold their job for a long time.
static LaunchCfg rule_cfg(bool small, uint64_t nshots, int nsm, bool shared_gpu, int nt_big) {
    if (small && (nshots > (uint64_t)nsm || shared_gpu)) return LaunchCfg{32, 24, 1, 0};
    if (shared_gpu) return LaunchCfg{128, 72, 1, 0};
    return LaunchCfg{nt_big, 200, 1, 0};
}

// Manual overrides for tuning and tests: QCMPS_ENGINE = warp | cta128 | cta256 | cta, QCMPS_SMEM_KB
// (work area per engine), QCMPS_WARPS (engines per CTA), QCMPS_BIG_KB (their shared area).  Returns true
// when any is set (the configuration is then not tuned).
static bool env_cfg(LaunchCfg& cfg, int nt_big) {
    bool any = false;
    if (const char* f = getenv("QCMPS_ENGINE")) {
        any = true;
        if (!strcmp(f, "warp")) cfg = LaunchCfg{32, 24, 1, 0};
        else if (!strcmp(f, "cta128")) cfg = LaunchCfg{128, 72, 1, 0};
        else if (!strcmp(f, "cta256")) cfg = LaunchCfg{256, 100, 1, 0};
        else if (!strcmp(f, "cta")) cfg = LaunchCfg{nt_big, 200, 1, 0};
    }
    if (const char* k = getenv("QCMPS_SMEM_KB")) { any = true; cfg.kb = atoi(k); }
    if (const char* w = getenv("QCMPS_WARPS")) { any = true; cfg.warps = atoi(w); }
    if (const char* b = getenv("QCMPS_BIG_KB")) { any = true; cfg.big_kb = atoi(b); }
    return any;
}

// Measured choice of the launch configuration (autotuner).  On the first batch of a (device, slot
// capacity, precision, size class) of a circuit, every candidate runs the shots' first eighth of the
// site-operation program on enough shots for about two rounds of its slots (results discarded), timed with
// CUDA events on the caller's stream; the configuration with the most shots per second is cached in the
// circuit and used from then on.  Candidates: for small capacities the warp variant at 16 / 20 / 24 / 28 /
// 32 KB and the 128- and 256-thread CTAs; for large capacities the 512-, 256- and 128-thread CTAs.
template <typename R, int NT_BIG>
static qc_status run_pass(CircuitImpl& c, EngineParams<R> P, const SlotLayout& L, const void* ref_state,
                          const int* cap_dev, const uint64_t* off_dev, const RefState& ref,
                          const uint64_t* shots_dev, uint64_t nshots, unsigned long long* counts_dev,
                          qc_shot_result* per_shot, cudaStream_t s, int max_slots, int nsm, bool defer,
                          LaunchCfg cfg);

template <typename R, int NT_BIG>
static LaunchCfg tuned_cfg(CircuitImpl& c, const EngineParams<R>& P, const SlotLayout& L, const void* ref_state,
                           const int* cap_dev, const uint64_t* off_dev, const RefState& ref, const uint64_t* shots_dev,
                           uint64_t nshots, cudaStream_t s, int nsm, int dev, bool small, LaunchCfg fallback) {
    const std::array<int, 4> key{dev, P.chi_max, P.precision, small ? 1 : 0};
    std::lock_guard<std::mutex> lk(c.tune_mu);
    auto it = c.tuned.find(key);
    if (it != c.tuned.end()) return LaunchCfg{it->second[0], it->second[1], 1, 0};
    std::vector<LaunchCfg> cand;
    if (small)
        cand = {{32, 16, 1, 0}, {32, 20, 1, 0}, {32, 24, 1, 0}, {32, 28, 1, 0}, {32, 32, 1, 0}, {128, 72, 1, 0},
                {256, 100, 1, 0}};
    else cand = {{NT_BIG, 200, 1, 0}, {256, 100, 1, 0}, {128, 72, 1, 0}};
    unsigned long long* scratch = nullptr;
    const size_t cb = 3 * (size_t)(P.wmax + 1) * sizeof(unsigned long long);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMallocAsync((void**)&scratch, cb, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (scratch) cudaFreeAsync(scratch, s);
        return fallback;
    }
    EngineParams<R> Pc = P;
    Pc.nops = std::max<uint32_t>(OPCH, P.nops / 8);
    Pc.per_shot = nullptr;
    Pc.trace_p1 = nullptr;
    Pc.trace_pos = nullptr;
    Pc.phase_cycles = nullptr;
    Pc.counts = scratch;
    const uint64_t tasks = std::min<uint64_t>(nshots, (small ? 18ull : 2ull) * (uint64_t)nsm);
    LaunchCfg best = fallback;
    double best_rate = -1.0;
    for (const LaunchCfg& cf : cand) {
        cudaEventRecord(e0, s);
        const qc_status st = run_pass<R, NT_BIG>(c, Pc, L, ref_state, cap_dev, off_dev, ref, shots_dev, tasks, scratch,
                                                 nullptr, s, 0, nsm, true, cf);
        cudaEventRecord(e1, s);
        float ms = 0;
        if (st != QC_OK || cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        const double rate = ms > 0 ? (double)tasks / ms : 0.0;
        if (rate > best_rate) {
            best_rate = rate;
            best = cf;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(scratch, s);
    c.tuned[key] = {best.variant, best.kb};
    return best;
}

// Host driver shared by mps_sample_batch and the serving loop.
//
// chi-bucketed variants: the reference run tells the bond dimensions the circuit reaches.  When
// they stay small (chi_peak <= 64, theta at most 128 x 128) every shot gets one warp of its own
// (NT = 32, many shot slots per SM, the common small updates latency-bound per warp); otherwise
// one CTA of NT_BIG threads works on each shot.
template <typename R, int NT_BIG>
static qc_status run_engine(CircuitImpl& c, qc_noise noise, const uint64_t* shots_dev, uint64_t nshots,
                            qc_mps_params prm, unsigned long long* counts_dev, int wmax,
                            qc_shot_result* per_shot, cudaStream_t s, int max_slots, bool shared_gpu,
                            qc_mps_trace* trace) {
    using V = typename VecOf<R>::T;
    DeviceCopy* dc;
    qc_status st = c.device_copy(&dc);
    if (st != QC_OK) return st;
    DeviceTables* tabs;
    st = device_tables(&tabs);
    if (st != QC_OK) return st;
    const SlotLayout L = slot_layout(c.n, prm.chi_max);
    const int chi = L.chi_cap;
    const uint64_t x_full = (uint64_t)(2 * chi + 1) * (2 * chi);
    const uint64_t over_full = (uint64_t)chi * chi * 3;
    const uint64_t xg_elems = std::max(x_full, over_full);
    // the same split scratch as the shots' slots (scratch_elems), including the room of an FP64 re-split
    const uint64_t scratch_stride = scratch_elems(chi, chi, sizeof(R), sizeof(V));

    int dev = 0, nsm = 0;
    QC_CUDA(cudaGetDevice(&dev));
    QC_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

    EngineParams<R> P{};
    P.chi_max = chi;
    P.chi_trunc = chi;
    P.shared_gpu = shared_gpu ? 1 : 0;
    P.prog = dc->mps;
    P.nops = (uint32_t)c.mps.size();
    P.nq = c.n;
    P.chan_kind = dc->chan_kind;
    P.nchan = (uint32_t)c.chan_kind.size();
    P.g1 = reinterpret_cast<const V*>(sizeof(R) == 4 ? (const void*)tabs->g1f : (const void*)tabs->g1d);
    P.g4 = reinterpret_cast<const V*>(sizeof(R) == 4 ? (const void*)tabs->g4f : (const void*)tabs->g4d);
    P.slot_stride = L.stride;
    P.scratch_stride = scratch_stride;
    P.xg_elems = xg_elems;
    P.cutoff = prm.cutoff;
    P.k0 = (uint32_t)noise.seed;
    P.k1 = (uint32_t)(noise.seed >> 32);
    const Thresholds th = make_thresholds(noise.p);
    for (int i = 0; i < 64; ++i) P.tg[i] = th.tg[i];
    P.weight = noise.fault_weight;
    P.tau = prm.tau;
    P.precision = prm.precision;
    P.wmax = wmax;
    P.sweep_cap = sizeof(R) == 4 ? 40 : 60;  // the noiseless reference run always keeps the default
    {
        int center = 0;
        for (const MpsOp& o : c.mps) {
            if (o.kind == M_G2) center = (o.flags & F_CENTER_RIGHT) ? o.q + 1 : o.q;
            else if (o.kind == M_MOVE) center = (o.flags & F_CENTER_RIGHT) ? o.q + 1 : o.q;
            else if (o.kind == M_MEAS || o.kind == M_RESET) center = o.q;
            else if (o.kind == M_PSWAP && (center == o.q || center == o.q + 1))
                center = (o.flags & F_PROD_LEFT) ? o.q : o.q + 1;
        }
        P.final_center = center;
    }

    // 1. the noiseless reference state, computed once per (device, chi_max, cutoff, precision)
    RefState* ref = nullptr;
    {
        std::lock_guard<std::mutex> lk(c.ref_mu);
        const RefKey key{dev, prm.chi_max, prm.precision, prm.cutoff};
        auto it = c.refs.find(key);
        if (it == c.refs.end()) {
            RefState rs;
            char* tmp = nullptr;
            const size_t tmp_bytes = scratch_stride * sizeof(V) + 64;
            cudaError_t e = cudaMalloc(&rs.state, L.stride * sizeof(V));
            if (e == cudaSuccess) e = cudaMalloc(&rs.dims, (c.n + 1) * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc(&rs.cap, (c.n + 1) * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc(&rs.off, (c.n + 1) * sizeof(uint64_t));
            if (e == cudaSuccess) e = cudaMallocAsync((void**)&tmp, tmp_bytes, s);
            if (e == cudaSuccess) e = cudaMemcpy(rs.cap, L.cap.data(), (c.n + 1) * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(rs.off, L.off.data(), (c.n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemsetAsync(tmp, 0, 64, s);
            qc_status out = QC_OK;
            if (e != cudaSuccess) out = cuda_fail(e, "reference workspace");
            if (out == QC_OK) {
                EngineParams<R> Pr = P;
                Pr.x_big = 0;
                const size_t smem = configure_smem<R, NT_BIG>(Pr, 200 * 1024, std::max(x_full, over_full));
                if (smem_optin((const void*)engine_kernel<R, NT_BIG>) != QC_OK) e = cudaErrorInvalidValue;
                Pr.reference = 1;
                Pr.mps = reinterpret_cast<V*>(rs.state);
                Pr.off = rs.off;
                Pr.ref_off = rs.off;
                Pr.ref_chi = chi;
                Pr.cap = rs.cap;
                Pr.scratch = reinterpret_cast<V*>(tmp + 64);
                Pr.ntasks = 1;
                Pr.next_task = reinterpret_cast<unsigned long long*>(tmp);
                Pr.ref_status = reinterpret_cast<int*>(tmp + 8);
                Pr.ref_chi_out = reinterpret_cast<int*>(tmp + 12);
                Pr.ref_disc_out = reinterpret_cast<double*>(tmp + 16);
                Pr.ref_dims_out = rs.dims;
                Pr.counts = nullptr;
                if (e == cudaSuccess) {
                    engine_kernel<R, NT_BIG><<<1, NT_BIG, smem, s>>>(Pr);
                    e = cudaGetLastError();
                }
                int st_h[2] = {0, 0};
                if (e == cudaSuccess) e = cudaMemcpyAsync(st_h, Pr.ref_status, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaMemcpyAsync(&rs.disc, Pr.ref_disc_out, sizeof(double), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e != cudaSuccess) out = cuda_fail(e, "reference run");
                else if (st_h[0] > 0) out = fail(QC_EINVAL, "measurement at instruction %d is not deterministically 0 in the noiseless circuit", st_h[0] - 1);
                else if (st_h[0] < 0) out = fail((qc_status)(st_h[0] + 1000), "reference run failed (status %d)", st_h[0] + 1000);
                rs.chi_peak = st_h[1];
                if (out == QC_OK) {
                    const int q = P.final_center;
                    std::vector<int> rd(c.n + 1);
                    e = cudaMemcpy(rd.data(), rs.dims, rd.size() * sizeof(int), cudaMemcpyDeviceToHost);
                    std::vector<V> cen;
                    if (e == cudaSuccess) {
                        cen.resize((size_t)rd[q] * 2 * rd[q + 1]);
                        e = cudaMemcpy(cen.data(), reinterpret_cast<V*>(rs.state) + L.off[q], cen.size() * sizeof(V),
                                       cudaMemcpyDeviceToHost);
                    }
                    if (e != cudaSuccess) out = cuda_fail(e, "reference centre");
                    double nn = 0;
                    for (const V& v : cen) nn += (double)v.x * v.x + (double)v.y * v.y;
                    rs.norm = nn;
                }
            }
            if (tmp) cudaFreeAsync(tmp, s);
            if (out != QC_OK) {
                cudaFree(rs.state); cudaFree(rs.dims); cudaFree(rs.cap); cudaFree(rs.off);
                return out;
            }
            it = c.refs.emplace(key, rs).first;
        }
        ref = &it->second;
    }
    if (nshots == 0) return QC_OK;
    if (trace && trace->sweep_cap > 0) P.sweep_cap = trace->sweep_cap;
    if (trace && trace->phase_cycles_dev) P.phase_cycles = reinterpret_cast<unsigned long long*>(trace->phase_cycles_dev);
    if (trace && trace->readout_p1_dev && trace->readout_k > 0) {
        P.trace_p1 = trace->readout_p1_dev;
        P.trace_k = trace->readout_k;
    }

    // 2. capacity bucket: slots sized for chi_alloc = min(chi, max(64, 2 chi_peak_ref)); a shot
    //    that outgrows it is reported by the first pass and re-run with full capacity
    const int chi_alloc = bucket_chi(ref->chi_peak, chi);
    const bool bucketed = chi_alloc < chi;
    // launch configuration: manual override, else the measured choice (batches that fill the GPU on
    // their own), else the rule
    // (the first pass is small when the noiseless run stays at bond 64, as most shots do; the re-run
    // pass holds exactly the shots that outgrew the bucket, so it is large)
    auto pick = [&](const EngineParams<R>& Pp, const SlotLayout& Lp, const int* cp, const uint64_t* op,
                    uint64_t n, bool first) {
        const bool small = first && ref->chi_peak <= 64;
        // the re-run pass (few shots, large theta) takes the largest CTA whether or not the GPU is shared
        LaunchCfg cf = first ? rule_cfg(small, n, nsm, shared_gpu, NT_BIG) : LaunchCfg{NT_BIG, 200, 1, 0};
        if (env_cfg(cf, NT_BIG)) {
            // the re-run pass holds the shots a one-warp engine cannot finish: never a warp
            if (!first && cf.variant == 32) cf = LaunchCfg{NT_BIG, 200, 1, 0};
            return cf;
        }
        if (first && !shared_gpu && n >= 2ull * (uint64_t)nsm && !getenv("QCMPS_NO_TUNE"))
            cf = tuned_cfg<R, NT_BIG>(c, Pp, Lp, ref->state, cp, op, *ref, shots_dev, n, s, nsm, dev, small, cf);
        return cf;
    };
    const SlotLayout L1 = bucketed ? slot_layout(c.n, chi_alloc) : L;
    int* cap1 = ref->cap;
    uint64_t* off1 = ref->off;
    if (bucketed) {
        std::lock_guard<std::mutex> lk(c.ref_mu);
        auto it = ref->packed.find(chi_alloc);
        if (it == ref->packed.end()) {
            RefPacked rp;  // the bucket's slot layout (the reference keeps its own)
            cudaError_t e = cudaMalloc(&rp.cap, (c.n + 1) * sizeof(int));
            if (e == cudaSuccess) e = cudaMalloc(&rp.off, (c.n + 1) * sizeof(uint64_t));
            if (e == cudaSuccess) e = cudaMemcpy(rp.cap, L1.cap.data(), (c.n + 1) * sizeof(int), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(rp.off, L1.off.data(), (c.n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) {
                cudaFree(rp.cap); cudaFree(rp.off);
                return cuda_fail(e, "bucket layout");
            }
            it = ref->packed.emplace(chi_alloc, rp).first;
        }
        cap1 = it->second.cap;
        off1 = it->second.off;
    }
    EngineParams<R> P1 = P;
    P1.chi_max = bucketed ? chi_alloc : chi;
    const LaunchCfg cf1 = pick(P1, L1, cap1, off1, nshots, true);
    if (trace) { trace->launch_threads_out = cf1.variant; trace->launch_kb_out = cf1.kb; }
    // one pass unless shots can be deferred: by the capacity bucket, or (complex64 in one warp per shot) by a
    // cut inside a cluster that needs the FP64 split
    if (!bucketed && !(sizeof(R) == 4 && cf1.variant == 32))
        return run_pass<R, NT_BIG>(c, P, L, ref->state, ref->cap, ref->off, *ref, shots_dev, nshots, counts_dev,
                                   per_shot, s, max_slots, nsm, false, cf1);
    // first pass: per-shot results are needed to find the shots to re-run
    qc_shot_result* res1 = per_shot;
    if (!res1) QC_CUDA(cudaMallocAsync((void**)&res1, nshots * sizeof(qc_shot_result), s));
    qc_status out = run_pass<R, NT_BIG>(c, P1, L1, ref->state, cap1, off1, *ref, shots_dev, nshots, counts_dev, res1,
                                        s, max_slots, nsm, true, cf1);
    std::vector<qc_shot_result> h;
    if (out == QC_OK) {
        h.resize(nshots);
        cudaError_t e = cudaMemcpyAsync(h.data(), res1, nshots * sizeof(qc_shot_result), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) out = cuda_fail(e, "first pass");
    }
    std::vector<uint64_t> redo, where;
    for (uint64_t i = 0; out == QC_OK && i < nshots; ++i)
        if (h[i].status == QC_ECAPACITY || h[i].status == QC_INTERNAL_FP64_RERUN) {
            redo.push_back(h[i].shot);
            where.push_back(i);
        }
    if (out == QC_OK && !redo.empty()) {
        // second pass with the full capacity, then the records go back to their places
        uint64_t* shots2 = nullptr;
        uint64_t* pos2 = nullptr;
        qc_shot_result* res2 = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&shots2, redo.size() * sizeof(uint64_t), s);
        if (e == cudaSuccess) e = cudaMallocAsync((void**)&res2, redo.size() * sizeof(qc_shot_result), s);
        if (e == cudaSuccess && P.trace_p1) e = cudaMallocAsync((void**)&pos2, where.size() * sizeof(uint64_t), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(shots2, redo.data(), redo.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && pos2)
            e = cudaMemcpyAsync(pos2, where.data(), where.size() * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) out = cuda_fail(e, "second pass");
        EngineParams<R> P2 = P;
        P2.trace_pos = pos2;
        // the re-run holds only the shots that outgrew the bucket: all of them run at once (its slots
        // are larger than the first pass's, so a caller's slot limit sized for those is not applied)
        if (out == QC_OK)
            out = run_pass<R, NT_BIG>(c, P2, L, ref->state, ref->cap, ref->off, *ref, shots2, redo.size(), counts_dev,
                                      res2, s, 0, nsm, false, pick(P2, L, ref->cap, ref->off, redo.size(), false));
        if (out == QC_OK && per_shot) {
            std::vector<qc_shot_result> h2(redo.size());
            e = cudaMemcpyAsync(h2.data(), res2, h2.size() * sizeof(qc_shot_result), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            for (size_t k = 0; e == cudaSuccess && k < where.size(); ++k)
                e = cudaMemcpyAsync(per_shot + where[k], &h2[k], sizeof(qc_shot_result), cudaMemcpyHostToDevice, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) out = cuda_fail(e, "second pass results");
        }
        cudaFreeAsync(shots2, s);
        cudaFreeAsync(res2, s);
        if (pos2) cudaFreeAsync(pos2, s);
    }
    if (res1 != per_shot) cudaFreeAsync(res1, s);
    return out;
}

// Argument checks of a sampling call (host only, before any device work).
static qc_status check_args(const CircuitImpl& c, qc_noise noise, const uint64_t* shots_dev, uint64_t nshots,
                            qc_mps_params prm) {
    if (!(noise.p >= 0.0 && noise.p < 1.0)) return fail(QC_EINVAL, "p must lie in [0, 1)");
    if (prm.chi_max < 1 || prm.chi_max > 1024) return fail(QC_EINVAL, "chi_max must be in [1, 1024]");
    if (!(prm.cutoff >= 0.0)) return fail(QC_EINVAL, "cutoff must be >= 0");
    if (prm.precision != QC_C64 && prm.precision != QC_C128) return fail(QC_EINVAL, "unknown precision");
    if (noise.fault_weight >= 0 && (uint64_t)noise.fault_weight > c.chan_kind.size())
        return fail(QC_EINVAL, "fault weight exceeds the number of channels");
    if (noise.fault_weight > MAXF) return fail(QC_EINVAL, "fault weight above %d", MAXF);
    if (nshots && !shots_dev) return fail(QC_EINVAL, "null shots");
    if (c.n < 2) return fail(QC_EINVAL, "the MPS engine needs at least two qubits");
    return QC_OK;
}

qc_status engine_launch(CircuitImpl& c, qc_noise noise, const uint64_t* shots_dev, uint64_t nshots,
                        qc_mps_params prm, unsigned long long* counts_dev, int wmax, qc_shot_result* per_shot,
                        cudaStream_t s, int max_slots, bool shared_gpu, qc_mps_trace* trace) {
    if (const qc_status a = check_args(c, noise, shots_dev, nshots, prm); a != QC_OK) return a;
    if (prm.precision == QC_C64)
        return run_engine<float, NT_F>(c, noise, shots_dev, nshots, prm, counts_dev, wmax, per_shot, s, max_slots,
                                       shared_gpu, trace);
    return run_engine<double, NT_D>(c, noise, shots_dev, nshots, prm, counts_dev, wmax, per_shot, s, max_slots,
                                    shared_gpu, trace);
}

qc_status shot_footprint(const CircuitImpl& c, qc_mps_params prm, uint64_t* bytes) {
    const SlotLayout L = slot_layout(c.n, std::max(1, prm.chi_max));
    const int chi = L.chi_cap;
    const bool c128 = prm.precision == QC_C128;
    const uint64_t es = c128 ? 16 : 8;
    *bytes = (L.stride + scratch_elems(chi, chi, c128 ? 8 : 4, es)) * es;
    return QC_OK;
}

}  // namespace qc

using namespace qc;

namespace qc {
qc_status bucket_footprint(CircuitImpl& c, qc_noise noise, qc_mps_params prm, cudaStream_t s, uint64_t* bytes) {
    // the reference run (cached) tells the bucket; nshots = 0 computes it and launches nothing else
    qc_status st = engine_launch(c, noise, nullptr, 0, prm, nullptr, 0, nullptr, s, 0, true);
    if (st != QC_OK) return st;
    int dev = 0;
    QC_CUDA(cudaGetDevice(&dev));
    int ref_chi = 1;
    {
        std::lock_guard<std::mutex> lk(c.ref_mu);
        auto it = c.refs.find(RefKey{dev, prm.chi_max, prm.precision, prm.cutoff});
        if (it == c.refs.end()) return fail(QC_EDEVICE, "reference state missing after the reference run");
        ref_chi = std::max(1, it->second.chi_peak);
    }
    const int chi = slot_layout(c.n, prm.chi_max).chi_cap;
    const int chi_alloc = bucket_chi(ref_chi, chi);
    const SlotLayout L1 = slot_layout(c.n, chi_alloc);
    const bool c128 = prm.precision == QC_C128;
    const uint64_t es = c128 ? 16 : 8;
    *bytes = (L1.stride + scratch_elems(chi_alloc, ref_chi, c128 ? 8 : 4, es)) * es;
    return QC_OK;
}
}  // namespace qc

extern "C" qc_status mps_sample_batch_traced(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                                             uint64_t nshots, qc_mps_params params, qc_counts* per_w, int32_t w_max,
                                             qc_shot_result* per_shot_dev, qc_mps_trace* trace, void* stream) {
    if (!circuit) return fail(QC_EINVAL, "null circuit");
    if (w_max < 0 || w_max > 4095) return fail(QC_EINVAL, "w_max must lie in [0, 4095]");
    if (trace && trace->readout_k < 0) return fail(QC_EINVAL, "readout_k must be >= 0");
    if (trace && trace->readout_k > 0 && nshots && !trace->readout_p1_dev)
        return fail(QC_EINVAL, "null readout record buffer");
    cudaStream_t s = (cudaStream_t)stream;
    CircuitImpl& c = const_cast<qc_circuit*>(circuit)->impl;
    if (const qc_status a = check_args(c, noise, shots_dev, nshots, params); a != QC_OK) return a;
    if (trace && trace->readout_p1_dev && trace->readout_k > 0 && nshots)  // all-ones bytes: NaN
        QC_CUDA(cudaMemsetAsync(trace->readout_p1_dev, 0xFF, nshots * (size_t)trace->readout_k * sizeof(double), s));
    unsigned long long* counts = nullptr;
    const size_t cb = 3 * (size_t)(w_max + 1) * sizeof(unsigned long long);
    QC_CUDA(cudaMallocAsync((void**)&counts, cb, s));
    qc_status st = QC_OK;
    cudaError_t e = cudaMemsetAsync(counts, 0, cb, s);
    if (e != cudaSuccess) st = cuda_fail(e, "memset");
    if (st == QC_OK)
        st = engine_launch(c, noise, shots_dev, nshots, params, counts, w_max, per_shot_dev, s, 0, false, trace);
    if (st == QC_OK) {
        std::vector<unsigned long long> h(3 * (w_max + 1));
        e = cudaMemcpyAsync(h.data(), counts, cb, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "engine");
        if (st == QC_OK && per_w)
            for (int w = 0; w <= w_max; ++w) {
                per_w[w].n += h[3 * w];
                per_w[w].n_acc += h[3 * w + 1];
                per_w[w].n_err += h[3 * w + 2];
            }
    }
    cudaFreeAsync(counts, s);
    return st;
}

extern "C" qc_status mps_sample_batch(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                                      uint64_t nshots, qc_mps_params params, qc_counts* per_w, int32_t w_max,
                                      qc_shot_result* per_shot_dev, void* stream) {
    return mps_sample_batch_traced(circuit, noise, shots_dev, nshots, params, per_w, w_max, per_shot_dev, nullptr,
                                   stream);
}

extern "C" qc_status mps_shot_footprint(const qc_circuit* circuit, qc_mps_params params, uint64_t* bytes) {
    if (!circuit || !bytes) return fail(QC_EINVAL, "null argument");
    return shot_footprint(circuit->impl, params, bytes);
}
