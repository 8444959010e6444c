// Internal declarations shared by the qcmps translation units.
#pragma once

#include <cuda_runtime.h>

#include <array>
#include <cstdint>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/qcmps.h"

namespace qc {

enum Kind : uint8_t {
    K_H, K_S, K_SDG, K_X, K_Y, K_Z, K_T, K_TDG, K_CX, K_CZ, K_SWAP, K_M, K_R, K_DEP1, K_DEP2, K_XERR
};

struct Op {
    uint8_t kind;
    int32_t q0, q1;
    uint32_t aux;  // channel id for noise, readout id for M/R
};

// ---- pre-screen program (one 8-byte word pair per frame-relevant instruction) ----------------
enum PreKind : uint32_t { P_H = 0, P_S, P_CX, P_CZ, P_SWAP, P_DEP1, P_DEP2, P_XERR, P_MDEC, P_CLEAR };
struct PreOp {
    uint32_t w0;  // kind | q0 << 4 | q1 << 16
    uint32_t w1;  // channel id
};
inline PreOp make_preop(uint32_t kind, uint32_t q0, uint32_t q1, uint32_t chan) {
    return PreOp{kind | (q0 << 4) | (q1 << 16), chan};
}

// ---- MPS program ---------------------------------------------------------------------------
enum MpsKind : uint8_t { M_G1 = 0, M_G2, M_CH1, M_CH2, M_MEAS, M_RESET, M_MOVE, M_PSWAP };
// F_PROD_LEFT: M_PSWAP whose product-state qubit sits on the left site of the pair
enum MpsFlag : uint8_t { F_CENTER_RIGHT = 1, F_POSTSELECT = 2, F_XERR = 4, F_PROD_LEFT = 8 };
struct MpsOp {
    uint8_t kind;
    uint8_t flags;
    uint16_t q;   // site (G1/CH/MEAS/RESET) or left site of the pair (G2)
    uint32_t a;   // gate index (G1: into the 2x2 table, G2: into the 4x4 table), channel (CH),
                  // readout id (MEAS/RESET)
    uint32_t b;   // CH2: second site
    int32_t src;  // instruction index in text order (for abort reporting), -1 if synthetic
};
static_assert(sizeof(MpsOp) == 16, "MpsOp layout");

// Gate table indices for the 2x2 table.
enum G1Index : uint32_t { G1_H = 0, G1_S, G1_SDG, G1_X, G1_Y, G1_Z, G1_T, G1_TDG, G1_COUNT };
// 4x4 table: CX(hi->lo), CX(lo->hi), CZ, SWAP, IDENTITY (centre moves)
enum G4Index : uint32_t { G4_CX_HL = 0, G4_CX_LH, G4_CZ, G4_SWAP, G4_ID, G4_COUNT };

struct DeviceCopy {
    PreOp* pre = nullptr;
    MpsOp* mps = nullptr;
    uint8_t* chan_kind = nullptr;  // per channel: 1 DEP1, 2 DEP2, 3 XERR
};

// Noiseless reference state cached per (device, chi_max, cutoff, precision).
struct RefKey {
    int device, chi_max, precision;
    double cutoff;
    bool operator<(const RefKey& o) const {
        if (device != o.device) return device < o.device;
        if (chi_max != o.chi_max) return chi_max < o.chi_max;
        if (precision != o.precision) return precision < o.precision;
        return cutoff < o.cutoff;
    }
};
struct RefPacked {  // the slot layout of a smaller capacity bucket
    void* state = nullptr;  // unused
    int* cap = nullptr;
    uint64_t* off = nullptr;
};
struct RefState {
    void* state = nullptr;     // one slot of site tensors
    int* dims = nullptr;       // [n+1] bond dimensions, device
    int* cap = nullptr;        // [n+1] bond capacities, device
    uint64_t* off = nullptr;   // [n+1] site offsets, device
    double disc = 0, norm = 0;
    int chi_peak = 0;
    std::map<int, RefPacked> packed;  // by slot capacity
};

struct CircuitImpl {
    int n = 0;
    std::vector<Op> ops;
    std::vector<uint8_t> chan_kind;
    std::vector<uint8_t> decided;  // per M instruction (text order)
    int64_t n_meas = 0, n_decided = 0, n_resets = 0, n_t = 0, n_readouts = 0;
    int64_t n_updates = 0;  // two-site updates and centre moves per shot
    int64_t n_pswaps = 0;   // SWAPs with a product-state qubit (no decomposition)
    std::vector<PreOp> pre;
    std::vector<MpsOp> mps;
    std::mutex mu;
    std::map<int, DeviceCopy> dev;  // per device
    std::mutex ref_mu;
    std::map<RefKey, RefState> refs;
    std::mutex tune_mu;
    std::map<std::array<int, 4>, std::array<int, 2>> tuned;  // (device, capacity, precision, small) -> launch
    ~CircuitImpl();
    // Upload the programs to the current device once; returns the device copy.
    qc_status device_copy(DeviceCopy** out);
};

// Error reporting (thread-local message).
qc_status fail(qc_status st, const char* fmt, ...);
qc_status cuda_fail(cudaError_t e, const char* what);
// Raise a kernel's dynamic shared-memory limit to the device's opt-in maximum, once per (device,
// kernel), so that concurrent launches with different sizes never race on the attribute.
qc_status smem_optin(const void* fn);
// The dynamic shared memory a launch of fn may ask for on the current device.
qc_status smem_limit(const void* fn, size_t* bytes);
#define QC_CUDA(call)                                         \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return ::qc::cuda_fail(e_, #call); \
    } while (0)

// Thresholds of the random-number contract.
struct Thresholds {
    uint32_t t1;
    uint32_t tg[64];
};
Thresholds make_thresholds(double p);

// Pre-screen and MPS engine drivers shared by the public entry points and the serving loop.
qc_status prescreen_run(CircuitImpl& c, qc_noise noise, uint64_t shot0, uint64_t nshots, uint64_t* kept_mask_dev,
                        qc_survivors* survivors, uint64_t* hist_drawn, uint64_t* hist_kept, int32_t w_max,
                        cudaStream_t s);
qc_status engine_launch(CircuitImpl& c, qc_noise noise, const uint64_t* shots_dev, uint64_t nshots,
                        qc_mps_params prm, unsigned long long* counts_dev, int wmax, qc_shot_result* per_shot,
                        cudaStream_t s, int max_slots, bool shared_gpu, qc_mps_trace* trace = nullptr);
qc_status shot_footprint(const CircuitImpl& c, qc_mps_params prm, uint64_t* bytes);
// Bytes of one shot slot of the first pass (the capacity bucket the engine allocates), computing and
// caching the noiseless reference state on `s` if needed.
qc_status bucket_footprint(CircuitImpl& c, qc_noise noise, qc_mps_params prm, cudaStream_t s, uint64_t* bytes);

// Pauli code conventions.
#if defined(__CUDACC__)
__host__ __device__
#endif
inline void pauli_xz(uint32_t p, uint32_t& x, uint32_t& z) {  // 0=I 1=X 2=Y 3=Z
    x = (p == 1 || p == 2);
    z = (p == 2 || p == 3);
}

}  // namespace qc

struct qc_circuit {
    qc::CircuitImpl impl;
};
