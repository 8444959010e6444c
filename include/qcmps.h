/*
 * qcmps — noisy-shot sampling of cultivation-shaped Clifford+T circuits on a B300 (sm_103a).
 *
 * C ABI of the library.  Every step of the sampling path runs in the library's own CUDA kernels;
 * the caller provides device memory and a CUDA stream.  All functions are thread-safe unless
 * stated otherwise.  Every function returns a qc_status; on failure qc_last_error() returns a
 * thread-local message and the outputs are unspecified.
 *
 * The problem statement follows Sec. 4 of "Comparing magic state cultivation methods using
 * matrix product states" (arXiv 2609.19116): a circuit of Clifford gates and T gates on a line
 * of qubits with Z measurements and resets; uniform depolarising noise of rate p (each of the
 * 4^k-1 non-identity Paulis of a k-qubit channel with probability p/(4^k-1)); a shot is kept only
 * if every measurement returns 0, and a kept shot is logically wrong when its final state's
 * squared overlap with the noiseless final state differs from 1 (Sec. 4, App. A.3).  Counts are
 * kept per fault weight w, the number of channels that fired (Sec. 4.1, Eq. estimators).
 *
 * Circuit text format: one instruction per line, '#' comments:
 *   QUBITS n | H q | S q | SDG q | X q | Y q | Z q | T q | TDG q | CX c t | CZ a b | SWAP a b |
 *   M q (Z measurement, post-selected on 0) | R q (reset to |0>) |
 *   DEP1 q | DEP2 a b (depolarising channels) | XERR q (X error channel) | TICK (no-op)
 * Noise channels are numbered 0.. in text order; readouts (M and R) likewise.
 *
 * Random numbers (Philox4x32-10, Salmon et al. SC'11; key = (seed mod 2^32, seed >> 32)):
 *   T1 = floor(p 2^32); y = 1 - T1/2^32; TG[s] = floor((1 - y^(s+1)) 2^32) for s = 0..63, the
 *   powers formed by successive FP64 multiplications.  Shots form 64-shot words w = shot >> 6.
 *   - channel c, word w: u = philox(c>>2, w, 0, 0)[c&3]; first faulted lane = min{s: u < TG[s]}
 *     (none if u >= TG[63]); further lanes by geometric skips from d_k = philox(c, w, k>>2, 1)[k&3],
 *     next lane = previous + 1 + min{s: d_k < TG[s]} while < 64.
 *   - Pauli of faulted lane j: x = philox(c, w, j, 2)[0]; code = 1 + (x*z >> 32), z = 3 (DEP1) or 15
 *     (DEP2, code i = (P_a, P_b) = (i>>2, i&3), 0=I 1=X 2=Y 3=Z); XERR is always X.
 *   - readout k of shot s: x = philox(k, s mod 2^32, s >> 32, 3); u = ((x0>>5) 2^26 + (x1>>6)) / 2^53;
 *     outcome 1 iff u < p1 (FP64).
 *   - fixed weight w (subset sampling, Sec. 4.1): Floyd's algorithm over the channels with draws
 *     philox(i, s mod 2^32, s >> 32, 4)[0] reduced to [0, j] by Lemire's multiply-shift with
 *     rejection; the Pauli of a chosen channel c from philox(c, s mod 2^32, s >> 32, 5)[0].
 */
#ifndef QCMPS_H
#define QCMPS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    QC_OK = 0,
    QC_PENDING = 1,      /* job not finished yet (mps_serve_poll) */
    QC_EINVAL = -1,      /* invalid argument or malformed circuit text */
    QC_ENOMEM = -2,      /* device or host allocation failed, or admission impossible */
    QC_EDEVICE = -3,     /* CUDA error */
    QC_ENOCONV = -4,     /* an SVD did not converge within its sweep limit */
    QC_ETIMEOUT = -5,    /* a bounded wait ran out */
    QC_ECANCELLED = -6,  /* job cancelled */
    QC_ECAPACITY = -7    /* a fixed-size buffer was too small (see the call's documentation) */
} qc_status;

/* Thread-local message describing the last failure of a call made on this thread. */
const char* qc_last_error(void);

/* ---- circuits --------------------------------------------------------------------------- */

typedef struct qc_circuit qc_circuit; /* opaque, owned by the library */

typedef struct {
    int32_t n_qubits;
    int64_t n_ops;           /* instructions other than QUBITS/TICK */
    int64_t n_channels;      /* noise channels M (Sec. 4.1) */
    int64_t n_measurements;  /* M instructions */
    int64_t n_decided;       /* measurements decided by stabiliser tracking (Sec. 4.2) */
    int64_t n_resets;
    int64_t n_t;             /* T and T^dagger gates */
    int64_t n_mps_updates;   /* two-site updates and centre moves per shot after SWAP routing */
    int64_t n_product_swaps; /* routing SWAPs with an unentangled qubit: exact, no decomposition */
} qc_circuit_info;

/* Parse circuit text (len bytes, need not be NUL-terminated).  Runs the offline analysis of
 * Sec. 4.2 (stabiliser tracking through diagonal non-Clifford gates; a measurement is decided
 * when +-Z_q is in the tracked group) and compiles the device programs.  *out is owned by the
 * library; release it with qc_circuit_free.  QC_EINVAL on malformed text. */
qc_status qc_circuit_parse(const char* text, size_t len, qc_circuit** out);
void qc_circuit_free(qc_circuit* circuit);
qc_status qc_circuit_get_info(const qc_circuit* circuit, qc_circuit_info* out);
/* flags[i] = 1 when the i-th M instruction (text order) is decided (Sec. 4.2).  Host buffer of
 * n_measurements bytes. */
qc_status qc_circuit_decided(const qc_circuit* circuit, uint8_t* flags);

/* ---- noise ---------------------------------------------------------------------------- */

typedef struct {
    double p;              /* uniform channel rate, 0 <= p < 1 (Sec. 4) */
    uint64_t seed;         /* Philox key */
    int32_t fault_weight;  /* -1: independent channels (Bernoulli p); w >= 0: exactly w faults */
} qc_noise;

/* Fault configurations of the given shots (Sec. 4: each channel resolves to a Pauli).
 * shots_dev: device array of nshots shot indices.  Outputs (device, caller-owned):
 * count_dev[i] = number of faults of shot i; chan_dev[i*max_faults + k], code_dev[...] its
 * faults sorted by channel (pauli code as in the header comment).  Shots with more than
 * max_faults faults have count_dev[i] = that number and only max_faults entries written.
 * Asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream). */
qc_status qc_sample_faults(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                           uint64_t nshots, uint32_t max_faults, uint32_t* count_dev,
                           uint32_t* chan_dev, uint8_t* code_dev, void* stream);

/* ---- pre-screen (Sec. 4.2) ----------------------------------------------------------- */

typedef struct {
    uint64_t* shots_dev;   /* caller-owned device buffer of `capacity` shot indices */
    uint64_t capacity;
    uint64_t count;        /* out: number of surviving shots (may exceed capacity; then only
                              the first `capacity`, in increasing order, are written) */
} qc_survivors;

/* Pauli-frame pre-screen of shots [shot0, shot0 + nshots) (shot0 a multiple of 64): per shot, the
 * fault configuration is propagated as a Pauli frame through the Clifford part (diagonal
 * non-Clifford gates leave it unchanged) and the shot is discarded when a decided measurement
 * flips; it never discards a shot that post-selection would keep (Sec. 4.2).
 *   kept_mask_dev  device, ceil(nshots/64) words; bit i of word k <-> shot shot0 + 64k + i
 *   survivors      optional (NULL): surviving shot indices, increasing
 *   hist_drawn, hist_kept  optional host arrays of w_max+1 counts: shots per fault weight w
 *                  (bin w_max collects w >= w_max), all drawn / surviving
 * Bernoulli noise (fault_weight = -1), or a fixed weight 0..32 (subset sampling, Sec. 4.1; up to
 * 128 qubits).  Synchronises `stream` before returning. */
qc_status pauli_prescreen(const qc_circuit* circuit, qc_noise noise, uint64_t shot0,
                          uint64_t nshots, uint64_t* kept_mask_dev, qc_survivors* survivors,
                          uint64_t* hist_drawn, uint64_t* hist_kept, int32_t w_max, void* stream);

/* The same pre-screen for callers that cannot allocate device memory: a process whose device
 * memory is a fixed pool owned by someone else, or an embedding runtime that forbids cudaMalloc.
 * (It is not for use inside a stream capture: it copies results to host memory and synchronises
 * the stream.)  The paper has no counterpart; it is a deployment convenience.  This entry point calls no cudaMalloc, cudaFree or
 * other allocating routine: its scratch (the staged frame program, the per-weight histograms and
 * the compaction offsets) lives in one file-scope device array of about 1.1 MB that every GPU
 * loading the library holds until the process exits.
 *   limits   at most 131072 frame-program words per circuit and 536,870,912 shots per call;
 *            larger requests return QC_ECAPACITY
 *   outputs  as pauli_prescreen: kept_mask_dev (ceil(nshots/64) words), survivors_dev (capacity
 *            shot indices, increasing), *n_kept (host; may exceed capacity), hist_drawn/hist_kept
 *            (optional host arrays of w_max+1 counts)
 *   set-up   the first call on a device looks up the array's device address
 *            (cudaGetSymbolAddress) with that device current; make that first call before any
 *            stream capture
 *   sharing  every call uses the same array and clears what must start at zero; calls whose work
 *            overlaps on the GPU (two streams, two host threads) race on it and must be serialised
 *            by the caller.  Synchronises `stream` before returning. */
qc_status pauli_prescreen_noalloc(const qc_circuit* circuit, qc_noise noise, uint64_t shot0,
                                  uint64_t nshots, uint64_t* kept_mask_dev, uint64_t* survivors_dev,
                                  uint64_t capacity, uint64_t* n_kept, uint64_t* hist_drawn,
                                  uint64_t* hist_kept, int32_t w_max, void* stream);

/* ---- batched MPS sampling (Sec. 3.1, 4, 4.3) --------------------------------------------- */

enum { QC_C64 = 0, QC_C128 = 1 };

typedef struct {
    int32_t chi_max;     /* bond dimension cap, 1 .. 1024 */
    double cutoff;       /* discarded-weight cutoff of the truncation rule */
    int32_t precision;   /* QC_C64: complex64 site tensors and SVD, FP64 probabilities and
                            discarded weight; QC_C128: complex128 throughout */
    double tau;          /* logical-error threshold on 1 - F; <= 0 selects 1e-8 (C128) or
                            max(1e-3, 10 * discarded weight) (C64) */
} qc_mps_params;

typedef struct { uint64_t n, n_acc, n_err; } qc_counts;

typedef struct {
    uint64_t shot;
    int32_t status;          /* 0 accepted, 1 rejected by a measurement, <0 a qc_status */
    int32_t weight;          /* fault weight w */
    int32_t logical_error;   /* accepted and 1 - F > tau */
    int32_t chi_peak;        /* largest bond kept during the shot */
    int64_t abort_op;        /* index (text order, instructions only) of the rejecting M, or -1 */
    double fidelity;         /* F = |<psi_ref|psi>|^2 / (<psi_ref|psi_ref><psi|psi>) */
    double discarded;        /* summed discarded weight of all truncations (FP64) */
    int32_t degenerate_cuts; /* truncations whose last kept and first dropped values tie */
    int32_t n_updates;       /* two-site updates performed */
    int32_t sweeps;          /* Jacobi sweeps summed over the shot's two-site updates */
    double alg_flops;        /* algorithmic real flops of the shot's two-site updates: contraction
                                8(2chi_l)chi_m(2chi_r), gate 128 chi_l chi_r, split by the R-SVD count
                                4(4 M^2 N + 22 N^3) (M >= N the sides of theta) plus the projection
                                8 r M N */
    int32_t gmem_updates;    /* two-site updates whose Jacobi matrix did not fit the engine's shared
                                memory and was rotated in global memory (blocked Jacobi) */
    int32_t fp64_resplits;   /* QC_C64: splits redone in FP64 because the truncation cut inside a cluster
                                of singular values that FP32 cannot tell apart and dropped more than the
                                cutoff's weight (a shot that meets one in a one-warp engine is re-run
                                from the start by a 512-thread engine, which counts them here) */
} qc_shot_result;

/* Simulate the given shots (typically pre-screen survivors) as MPS: single-site gates in place;
 * a two-site gate contracts the pair, applies the 4x4 gate and splits by SVD, keeping the
 * smallest count of singular values whose discarded tail sum s_i^2 is <= cutoff * sum s_i^2,
 * at most chi_max, renormalised (Sec. 3.1; the truncation rule itself is not fixed by the
 * paper, which runs untruncated); SWAP routing for non-adjacent pairs (Sec. 3.1); a measurement
 * samples the orthogonality-centre marginal in FP64, projects, renormalises and ends the shot
 * when it returns 1 (Sec. 4.3).  At the end F is formed against the noiseless reference state.
 *   shots_dev      device array of nshots shot indices
 *   per_w          host array of w_max+1 counts, ACCUMULATED into (bin w_max collects w >= w_max):
 *                  n = simulated shots, n_acc = accepted, n_err = accepted with a logical error
 *   per_shot_dev   optional device array of nshots results
 * Engines: one warp per shot for circuits whose noiseless run stays at bond 64, else one CTA per
 * shot, in slots of a capacity bucket; shots that outgrow the bucket (or need an FP64 re-split in a
 * one-warp engine) are re-run at full capacity in a second launch, their records replaced.
 * Synchronises `stream` before returning.  QC_EINVAL for chi_max outside [1, 1024], a negative
 * cutoff, an unknown precision, or a noiseless circuit with a measurement that is not
 * deterministically 0 (the argument checks come before any device work).  Per-shot failures are
 * reported in per_shot_dev status. */
qc_status mps_sample_batch(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                           uint64_t nshots, qc_mps_params params, qc_counts* per_w,
                           int32_t w_max, qc_shot_result* per_shot_dev, void* stream);

/* Verification hooks of mps_sample_batch (the paper has no counterpart; they exist so that tests can
 * compare intermediate quantities with a reference simulator and exercise the bounded limits).
 *   readout_p1_dev  optional device array of nshots x readout_k doubles, row i for shots_dev[i]:
 *                   column k = the Born probability of outcome 1 (FP64) of the shot's readout k
 *                   (M and R instructions numbered in text order); NaN where the shot ended before
 *                   reaching readout k.  Caller-owned; filled by the call.
 *   readout_k       columns of readout_p1_dev (0 = no record)
 *   sweep_cap       > 0: Jacobi sweep limit of every split of the shots (default 40 for QC_C64, 60
 *                   for QC_C128); a split that does not converge within it ends its shot with
 *                   per-shot status QC_ENOCONV.  The noiseless reference run keeps the default.
 *   phase_cycles_dev  optional device array of 8 counters, ACCUMULATED into: SM clock cycles spent
 *                   by the shots' engines in each phase (summed over engines): 0 fault draws,
 *                   1 two-site update up to the SVD (staging, gate fusion, contraction), 2 Jacobi,
 *                   3 spectrum, truncation and the write-back of both factors, 4 centre moves,
 *                   5 product-state SWAPs, 6 readouts, 7 the final overlap and the counters.
 *   launch_threads_out, launch_kb_out  out: the launch configuration of the (first) pass -- threads
 *                   per shot (32 = one warp per shot) and the work area per shot in KB -- as chosen by
 *                   the library's autotuner, its rule or the QCMPS_* overrides. */
typedef struct {
    double* readout_p1_dev;
    int32_t readout_k;
    int32_t sweep_cap;
    uint64_t* phase_cycles_dev;
    int32_t launch_threads_out;
    int32_t launch_kb_out;
} qc_mps_trace;

/* mps_sample_batch with the verification hooks above (trace may be NULL, which is mps_sample_batch). */
qc_status mps_sample_batch_traced(const qc_circuit* circuit, qc_noise noise, const uint64_t* shots_dev,
                                  uint64_t nshots, qc_mps_params params, qc_counts* per_w,
                                  int32_t w_max, qc_shot_result* per_shot_dev,
                                  qc_mps_trace* trace, void* stream);

/* Bytes of device memory one in-flight shot needs (site tensors at their capacities plus the
 * per-shot split scratch), the footprint used for admission. */
qc_status mps_shot_footprint(const qc_circuit* circuit, qc_mps_params params, uint64_t* bytes);

/* ---- measurement support (no counterpart in the paper) -------------------------------------- */

/* Issue rates of the current device's arithmetic units, the denominators of the rooflines of the
 * MPS engine (FP32) and of the pre-screen (32-bit integer logic).  Each rate comes from a kernel of
 * long independent chains of one instruction on every SM (4 CTAs x 256 threads per SM, 8 chains per
 * thread), the best of three launches timed with CUDA events on `stream`; it takes ~50 ms.
 *   ffma_tflops   FP32 fused multiply-add, 2 flops each
 *   ffma2_tflops  paired FP32 fused multiply-add (two lanes of a 64-bit register), 4 flops each
 *   dfma_tflops   FP64 fused multiply-add, 2 flops each
 *   lop3_tops     32-bit three-input logic operations (1e12 per second)
 *   imad_tops     32-bit integer multiply-adds (1e12 per second)
 *   sm_count, sm_clock_mhz  from the device attributes (the clock is the maximum SM clock) */
typedef struct {
    int32_t sm_count;
    double sm_clock_mhz;
    double ffma_tflops, ffma2_tflops, dfma_tflops, lop3_tops, imad_tops;
} qc_alu_peaks;
qc_status qc_measure_alu_peaks(qc_alu_peaks* out, void* stream);

/* ---- serving loop ---------------------------------------------------------------------- */

typedef struct qc_server qc_server;

typedef struct {
    uint64_t hbm_budget_bytes;  /* admission budget for in-flight MPS state */
    int32_t max_slots;          /* upper bound on the shot slots of one batch (0 = 16 x SMs) */
    int32_t n_streams;          /* device streams the loop spreads jobs over (0 = default 64) */
} qc_serve_cfg;

typedef struct {
    int32_t state;              /* QC_OK done, QC_PENDING running/queued, or an error status */
    uint64_t shots;             /* shots drawn */
    uint64_t survivors;         /* shots kept by the pre-screen */
    qc_counts counts[16];       /* per fault weight, bin 15 collects w >= 15 */
    double submit_ms, start_ms, end_ms; /* on the server's clock */
    char error[224];            /* when state < 0: the failing call's message (NUL-terminated) */
} qc_job_result;

/* Start a request loop on the current device.  Jobs are pre-screened as they arrive; their
 * surviving shots are cut into chunks of at most 512 shots, and n_streams worker threads each
 * launch one chunk at a time as its own persistent engine batch on their own stream, so chunks
 * of different jobs overlap on the device (each batch holds the shots of one job; inside it a
 * finished shot slot is back-filled with the next shot).  A chunk is launched only while its
 * footprint (slots x bytes of one slot of the capacity bucket the engine allocates) fits the
 * budget next to the chunks in flight; a chunk granted fewer slots than it has shots shrinks to two
 * shots per slot (the rest of the job waits for memory).  The re-run of a chunk's shots that outgrew
 * the bucket, at full capacity, is not charged: it can exceed the budget by its shots x one
 * full-capacity slot.  Chunks go to the job with the smallest remaining work
 * divided by 1 + age/1 s (age since submission); jobs older than 2 s go first, oldest first.
 * *out is owned by the library; release with mps_serve_destroy. */
qc_status mps_serve_create(const qc_serve_cfg* cfg, qc_server** out);
/* Queue nshots shots [shot0, shot0 + nshots) of a circuit (shot0 a multiple of 64).  The circuit
 * must stay alive until the job is done or cancelled. */
qc_status mps_serve_submit(qc_server* server, const qc_circuit* circuit, qc_noise noise,
                           qc_mps_params params, uint64_t shot0, uint64_t nshots,
                           uint64_t* job_id);
/* QC_PENDING while the job runs; QC_OK with *out filled when done. */
qc_status mps_serve_poll(qc_server* server, uint64_t job_id, qc_job_result* out);
qc_status mps_serve_cancel(qc_server* server, uint64_t job_id);
/* Stops the loop (cancelling queued jobs) and frees everything. */
void mps_serve_destroy(qc_server* server);

#ifdef __cplusplus
}
#endif

#endif /* QCMPS_H */
