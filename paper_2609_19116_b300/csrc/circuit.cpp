// Circuit parsing, the offline stabiliser analysis (Sec. 4.2) and compilation of the device
// programs: the Pauli-frame program of the pre-screen and the site-operation program of the MPS
// engine (SWAP routing, Sec. 3.1, and orthogonality-centre planning).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <set>
#include <sstream>

#include "qc_internal.h"

namespace qc {

static thread_local std::string g_last_error;

qc_status fail(qc_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

qc_status cuda_fail(cudaError_t e, const char* what) {
    return fail(QC_EDEVICE, "%s: %s", what, cudaGetErrorString(e));
}

// A kernel's dynamic shared-memory limit is process-wide state of the device.  Setting it per call to
// the size that call needs races with concurrent callers (a host thread that lowers it between another
// thread's set and launch makes that launch fail), so it is raised once per (device, kernel) to the
// device's opt-in maximum and never lowered; every launch then only asks for what it needs.
qc_status smem_optin(const void* fn) {
    static std::mutex mu;
    static std::set<std::pair<int, const void*>> done;
    int d = 0;
    QC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(mu);
    if (done.count({d, fn})) return QC_OK;
    int optin = 0;
    QC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d));
    cudaFuncAttributes fa{};
    QC_CUDA(cudaFuncGetAttributes(&fa, fn));
    const int dyn = optin - (int)fa.sharedSizeBytes;
    QC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    done.insert({d, fn});
    return QC_OK;
}

qc_status smem_limit(const void* fn, size_t* bytes) {
    int d = 0;
    QC_CUDA(cudaGetDevice(&d));
    int optin = 0;
    QC_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d));
    cudaFuncAttributes fa{};
    QC_CUDA(cudaFuncGetAttributes(&fa, fn));
    *bytes = (size_t)(optin - (int)fa.sharedSizeBytes);
    return QC_OK;
}

Thresholds make_thresholds(double p) {
    Thresholds t{};
    double f = std::floor(p * 4294967296.0);
    t.t1 = f >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)f;
    const double y = 1.0 - (double)t.t1 / 4294967296.0;
    double ys = y;
    for (int s = 0; s < 64; ++s) {
        double v = std::floor((1.0 - ys) * 4294967296.0);
        t.tg[s] = v >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)v;
        ys = ys * y;
    }
    return t;
}

// ---- offline stabiliser analysis (Sec. 4.2) --------------------------------------------------
// Rows are Pauli shapes [x | z] over n qubits, W 64-bit words each half.
namespace {
struct Group {
    int n, W;
    std::vector<std::vector<uint64_t>> rows;  // each 2W words
    explicit Group(int n_) : n(n_), W((n_ + 63) / 64) {
        for (int q = 0; q < n; ++q) {
            std::vector<uint64_t> r(2 * W, 0);
            r[W + q / 64] |= 1ull << (q % 64);
            rows.push_back(r);
        }
    }
    static bool get(const std::vector<uint64_t>& r, int bit) { return (r[bit / 64] >> (bit % 64)) & 1; }
    static void put(std::vector<uint64_t>& r, int bit, bool v) {
        uint64_t m = 1ull << (bit % 64);
        if (v) r[bit / 64] |= m; else r[bit / 64] &= ~m;
    }
    bool xq(const std::vector<uint64_t>& r, int q) const { return get(r, q); }
    bool zq(const std::vector<uint64_t>& r, int q) const { return get(r, W * 64 + q); }
    void setx(std::vector<uint64_t>& r, int q, bool v) const { put(r, q, v); }
    void setz(std::vector<uint64_t>& r, int q, bool v) const { put(r, W * 64 + q, v); }

    void conj(uint8_t kind, int a, int b) {
        for (auto& r : rows) {
            switch (kind) {
                case K_H: { bool x = xq(r, a), z = zq(r, a); setx(r, a, z); setz(r, a, x); break; }
                case K_S: case K_SDG: setz(r, a, zq(r, a) ^ xq(r, a)); break;
                case K_CX: setx(r, b, xq(r, b) ^ xq(r, a)); setz(r, a, zq(r, a) ^ zq(r, b)); break;
                case K_CZ: { bool xa = xq(r, a), xb = xq(r, b);
                             setz(r, a, zq(r, a) ^ xb); setz(r, b, zq(r, b) ^ xa); break; }
                case K_SWAP: { bool xa = xq(r, a), za = zq(r, a);
                               setx(r, a, xq(r, b)); setz(r, a, zq(r, b)); setx(r, b, xa); setz(r, b, za); break; }
                default: break;
            }
        }
    }
    // Keep the subgroup whose elements have no X component on qubit q.
    void drop_x_on(int q) {
        int piv = -1;
        for (size_t i = 0; i < rows.size(); ++i)
            if (xq(rows[i], q)) { piv = (int)i; break; }
        if (piv < 0) return;
        for (size_t i = piv + 1; i < rows.size(); ++i)
            if (xq(rows[i], q))
                for (int k = 0; k < 2 * W; ++k) rows[i][k] ^= rows[piv][k];
        rows.erase(rows.begin() + piv);
    }
    // Is the shape v in the span of the rows?  (Gaussian elimination over GF(2).)
    bool in_span(std::vector<uint64_t> v) const {
        std::vector<std::vector<uint64_t>> m = rows;
        const int nb = 2 * W * 64;
        size_t rank = 0;
        for (int bit = 0; bit < nb && rank < m.size(); ++bit) {
            size_t p = rank;
            while (p < m.size() && !get(m[p], bit)) ++p;
            if (p == m.size()) continue;
            std::swap(m[p], m[rank]);
            for (size_t i = 0; i < m.size(); ++i)
                if (i != rank && get(m[i], bit))
                    for (int k = 0; k < 2 * W; ++k) m[i][k] ^= m[rank][k];
            if (get(v, bit))
                for (int k = 0; k < 2 * W; ++k) v[k] ^= m[rank][k];
            ++rank;
        }
        for (int k = 0; k < 2 * W; ++k)
            if (v[k]) return false;
        return true;
    }
    std::vector<uint64_t> z_row(int q) const {
        std::vector<uint64_t> r(2 * W, 0);
        r[W + q / 64] |= 1ull << (q % 64);
        return r;
    }
    bool contains_z(int q) const { return in_span(z_row(q)); }
    void add_z(int q) {
        if (!contains_z(q)) rows.push_back(z_row(q));
    }
};

bool is_clifford_conj(uint8_t k) {
    return k == K_H || k == K_S || k == K_SDG || k == K_CX || k == K_CZ || k == K_SWAP;
}
}  // namespace

static void analyse(CircuitImpl& c) {
    Group g(c.n);
    c.decided.clear();
    for (const Op& op : c.ops) {
        switch (op.kind) {
            case K_T: case K_TDG: g.drop_x_on(op.q0); break;
            case K_M: {
                bool d = g.contains_z(op.q0);
                c.decided.push_back(d ? 1 : 0);
                g.drop_x_on(op.q0);
                g.add_z(op.q0);
                break;
            }
            case K_R: g.drop_x_on(op.q0); g.add_z(op.q0); break;
            default:
                if (is_clifford_conj(op.kind)) g.conj(op.kind, op.q0, op.q1);
                break;
        }
    }
}

// ---- pre-screen program ----------------------------------------------------------------------
static void compile_prescreen(CircuitImpl& c) {
    c.pre.clear();
    size_t mi = 0;
    for (const Op& op : c.ops) {
        switch (op.kind) {
            case K_H: c.pre.push_back(make_preop(P_H, op.q0, 0, 0)); break;
            case K_S: case K_SDG: c.pre.push_back(make_preop(P_S, op.q0, 0, 0)); break;
            case K_CX: c.pre.push_back(make_preop(P_CX, op.q0, op.q1, 0)); break;
            case K_CZ: c.pre.push_back(make_preop(P_CZ, op.q0, op.q1, 0)); break;
            case K_SWAP: c.pre.push_back(make_preop(P_SWAP, op.q0, op.q1, 0)); break;
            case K_DEP1: c.pre.push_back(make_preop(P_DEP1, op.q0, 0, op.aux)); break;
            case K_DEP2: c.pre.push_back(make_preop(P_DEP2, op.q0, op.q1, op.aux)); break;
            case K_XERR: c.pre.push_back(make_preop(P_XERR, op.q0, 0, op.aux)); break;
            case K_M:
                c.pre.push_back(make_preop(c.decided[mi++] ? P_MDEC : P_CLEAR, op.q0, 0, 0));
                break;
            case K_R: c.pre.push_back(make_preop(P_CLEAR, op.q0, 0, 0)); break;
            default: break;  // X, Y, Z, T, TDG leave the frame unchanged
        }
    }
}

// ---- MPS program ------------------------------------------------------------------------------
namespace {
struct SiteOp {
    uint8_t kind;
    uint8_t flags;
    int q;
    uint32_t a, b;
    int32_t src;
};
}  // namespace

static uint32_t g1_index(uint8_t k) {
    switch (k) {
        case K_H: return G1_H; case K_S: return G1_S; case K_SDG: return G1_SDG;
        case K_X: return G1_X; case K_Y: return G1_Y; case K_Z: return G1_Z;
        case K_T: return G1_T; default: return G1_TDG;
    }
}

// Execution order and SWAP routing of the instructions for the MPS engine.
//
// Order.  Instructions on disjoint qubits commute, so the order may follow the orthogonality
// centre instead of the text: a greedy list schedule over the dependency graph (each qubit's
// instructions stay in text order) that always takes the ready instruction closest to the centre.
// Readouts (M and R) also stay in text order among themselves, so every readout sees the same
// earlier projections as in text order and a shot's sampled outcomes do not depend on the schedule.
//
// Routing (Sec. 3.1: gates between qubits that are not neighbours on the line go through SWAPs).
// The line holds a permutation of the logical qubits.  A two-qubit gate at line distance d > 1
// moves one of its qubits next to the other with d - 1 adjacent SWAPs and leaves it there instead
// of swapping it back.  The qubit that moves is, in this order: the one in a product state (its
// SWAPs need no decomposition, see below); the one whose next reset comes first (an ancilla, which
// walks home after that reset); the one whose next partner lies closer to where it would land.
// A logical SWAP gate only exchanges the two labels.
//
// Product states are known at compile time: a qubit is unentangled from its last readout (which
// leaves it in |0>) or from the start until its next entangling gate, since single-qubit gates and
// Pauli faults keep it so.  Its site tensor is then |0> x M with the single-qubit gates since the
// readout still pending, and a SWAP with it is a relabelling of bonds (M_PSWAP), exact and cheap.
// After a reset the qubit walks back to its home site that way.
static void compile_mps(CircuitImpl& c) {
    const size_t N = c.ops.size();
    const int n = c.n;
    // dependency graph
    std::vector<std::vector<uint32_t>> succ(N);
    std::vector<int> indeg(N, 0);
    {
        std::vector<long> last_q(n, -1);
        long last_read = -1;
        for (size_t i = 0; i < N; ++i) {
            const Op& op = c.ops[i];
            long deps[3] = {last_q[op.q0], op.q1 >= 0 ? last_q[op.q1] : -1,
                            (op.kind == K_M || op.kind == K_R) ? last_read : -1};
            for (int a = 0; a < 3; ++a) {
                if (deps[a] < 0) continue;
                bool dup = false;
                for (int b = 0; b < a; ++b) dup |= deps[b] == deps[a];
                if (dup) continue;
                succ[deps[a]].push_back((uint32_t)i);
                ++indeg[i];
            }
            last_q[op.q0] = (long)i;
            if (op.q1 >= 0) last_q[op.q1] = (long)i;
            if (op.kind == K_M || op.kind == K_R) last_read = (long)i;
        }
    }
    // per qubit, text positions of its resets and of its two-qubit gates (for the mover choice)
    std::vector<std::vector<uint32_t>> resets(n), gates2(n);
    for (size_t i = 0; i < N; ++i) {
        const Op& op = c.ops[i];
        if (op.kind == K_R) resets[op.q0].push_back((uint32_t)i);
        if (op.kind == K_CX || op.kind == K_CZ || op.kind == K_SWAP) {
            gates2[op.q0].push_back((uint32_t)i);
            gates2[op.q1].push_back((uint32_t)i);
        }
    }
    auto next_after = [](const std::vector<uint32_t>& v, size_t i) -> long {
        auto it = std::upper_bound(v.begin(), v.end(), (uint32_t)i);
        return it == v.end() ? -1 : (long)*it;
    };
    std::vector<int> pos(n), at(n);
    std::vector<char> prod(n, 1);
    for (int q = 0; q < n; ++q) pos[q] = at[q] = q;

    std::vector<SiteOp> s;
    auto emit_swap = [&](int k) {  // exchange the qubits on sites k and k+1
        const int x = at[k], y = at[k + 1];
        if (prod[x] || prod[y]) s.push_back({M_PSWAP, (uint8_t)(prod[x] ? F_PROD_LEFT : 0), k, 0, 0, -1});
        else s.push_back({M_G2, 0, k, G4_SWAP, 0, -1});
        at[k] = y; at[k + 1] = x;
        pos[x] = k + 1; pos[y] = k;
    };
    auto needs_center = [&](const Op& op) {
        return op.kind == K_CX || op.kind == K_CZ || op.kind == K_M || op.kind == K_R;
    };
    std::vector<uint32_t> ready;
    for (size_t i = 0; i < N; ++i)
        if (indeg[i] == 0) ready.push_back((uint32_t)i);
    int center = 0;
    while (!ready.empty()) {
        // instructions that need no centre go first (lowest text index), else the nearest one
        size_t best = 0;
        long best_key = -1;
        for (size_t k = 0; k < ready.size(); ++k) {
            const Op& op = c.ops[ready[k]];
            long dist = 0;
            if (needs_center(op)) {
                const int p0 = pos[op.q0], p1 = op.q1 >= 0 ? pos[op.q1] : p0;
                const int lo = std::min(p0, p1), hi = std::max(p0, p1);
                dist = 1 + (center < lo ? lo - center : center > hi ? center - hi : 0);
            }
            const long key = dist * (long)(N + 1) + (long)ready[k];
            if (best_key < 0 || key < best_key) { best_key = key; best = k; }
        }
        const uint32_t i = ready[best];
        ready[best] = ready.back();
        ready.pop_back();
        const Op& op = c.ops[i];
        const int32_t src = (int32_t)i;
        switch (op.kind) {
            case K_H: case K_S: case K_SDG: case K_X: case K_Y: case K_Z: case K_T: case K_TDG:
                s.push_back({M_G1, 0, pos[op.q0], g1_index(op.kind), 0, src});
                break;
            case K_SWAP: {  // relabel
                const int a = op.q0, b = op.q1;
                std::swap(pos[a], pos[b]);
                at[pos[a]] = a;
                at[pos[b]] = b;
                std::swap(prod[a], prod[b]);
                break;
            }
            case K_CX: case K_CZ: {
                const int a = op.q0, b = op.q1;
                int mv;
                if (prod[a] != prod[b]) {
                    mv = prod[a] ? a : b;
                } else {
                    const long ra = next_after(resets[a], i), rb = next_after(resets[b], i);
                    if (ra != rb && (ra >= 0 || rb >= 0)) {
                        mv = (rb < 0 || (ra >= 0 && ra < rb)) ? a : b;
                    } else {
                        auto score = [&](int m_, int o_) {
                            const int d = std::abs(pos[m_] - pos[o_]) - 1;
                            const int dest = pos[m_] < pos[o_] ? pos[o_] - 1 : pos[o_] + 1;
                            double sc = d;
                            const long j = next_after(gates2[m_], i);
                            if (j >= 0) {
                                const Op& nx = c.ops[j];
                                const int partner = nx.q0 == m_ ? nx.q1 : nx.q0;
                                if (partner != o_) sc += 0.5 * std::max(0, std::abs(dest - pos[partner]) - 1);
                            }
                            return sc;
                        };
                        mv = score(a, b) <= score(b, a) ? a : b;
                    }
                }
                const int other = mv == a ? b : a;
                while (std::abs(pos[mv] - pos[other]) > 1) emit_swap(pos[mv] < pos[other] ? pos[mv] : pos[mv] - 1);
                const int left = std::min(pos[a], pos[b]);
                uint32_t g;
                if (op.kind == K_CX) g = (pos[a] == left) ? G4_CX_HL : G4_CX_LH;
                else g = G4_CZ;
                s.push_back({M_G2, 0, left, g, 0, src});
                prod[a] = prod[b] = 0;
                break;
            }
            case K_DEP1: s.push_back({M_CH1, 0, pos[op.q0], op.aux, 0, src}); break;
            case K_XERR: s.push_back({M_CH1, F_XERR, pos[op.q0], op.aux, 0, src}); break;
            case K_DEP2: s.push_back({M_CH2, 0, pos[op.q0], op.aux, (uint32_t)pos[op.q1], src}); break;
            case K_M:
                s.push_back({M_MEAS, F_POSTSELECT, pos[op.q0], op.aux, 0, src});
                prod[op.q0] = 1;
                break;
            case K_R: {
                const int q = op.q0;
                s.push_back({M_RESET, 0, pos[q], op.aux, 0, src});
                prod[q] = 1;
                while (pos[q] != q) emit_swap(pos[q] > q ? pos[q] - 1 : pos[q]);
                break;
            }
            default: break;
        }
        if (needs_center(op)) {
            const int p0 = pos[op.q0], p1 = op.q1 >= 0 ? pos[op.q1] : p0;
            const int lo = std::min(p0, p1), hi = std::max(p0, p1);
            center = center < lo ? lo : (center > hi ? hi : center);
        }
        for (uint32_t sx : succ[i])
            if (--indeg[sx] == 0) ready.push_back(sx);
    }

    // centre planning: each G2 needs the centre on one of its sites, each readout on its site;
    // after a G2 the centre goes to the side of the next site that needs it.  A product SWAP needs
    // no centre; when the centre is on its pair it ends on the entangled qubit's new site.
    const size_t NS = s.size();
    std::vector<int> next_need(NS + 1, -1);  // position (site) of the next centre-needing op
    for (size_t i = NS; i-- > 0;) {
        next_need[i] = next_need[i + 1];
        if (s[i].kind == M_G2) next_need[i] = s[i].q;  // pair (q, q+1)
        else if (s[i].kind == M_MEAS || s[i].kind == M_RESET) next_need[i] = s[i].q;
    }
    c.mps.clear();
    center = 0;
    auto move_to = [&](int t) {
        while (center < t) {
            c.mps.push_back({M_MOVE, F_CENTER_RIGHT, (uint16_t)center, 0, 0, -1});
            ++center;
        }
        while (center > t) {
            c.mps.push_back({M_MOVE, 0, (uint16_t)(center - 1), 0, 0, -1});
            --center;
        }
    };
    for (size_t i = 0; i < NS; ++i) {
        const SiteOp& o = s[i];
        if (o.kind == M_G2) {
            if (center < o.q) move_to(o.q);
            else if (center > o.q + 1) move_to(o.q + 1);
            const int nx = next_need[i + 1];
            const bool right = (nx < 0) ? true : (nx > o.q);
            c.mps.push_back({M_G2, (uint8_t)(right ? F_CENTER_RIGHT : 0), (uint16_t)o.q, o.a, 0, o.src});
            center = right ? o.q + 1 : o.q;
        } else if (o.kind == M_PSWAP) {
            c.mps.push_back({M_PSWAP, o.flags, (uint16_t)o.q, 0, 0, -1});
            if (center == o.q || center == o.q + 1) center = (o.flags & F_PROD_LEFT) ? o.q : o.q + 1;
        } else if (o.kind == M_MEAS || o.kind == M_RESET) {
            move_to(o.q);
            c.mps.push_back({o.kind, o.flags, (uint16_t)o.q, o.a, 0, o.src});
        } else {
            c.mps.push_back({o.kind, o.flags, (uint16_t)o.q, o.a, o.b, o.src});
        }
    }
    c.n_updates = 0;
    c.n_pswaps = 0;
    for (const MpsOp& m : c.mps) {
        c.n_updates += (m.kind == M_G2 || m.kind == M_MOVE);
        c.n_pswaps += m.kind == M_PSWAP;
    }
}

CircuitImpl::~CircuitImpl() {
    for (auto& kv : dev) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(kv.first);
        cudaFree(kv.second.pre);
        cudaFree(kv.second.mps);
        cudaFree(kv.second.chan_kind);
        cudaSetDevice(cur);
    }
    for (auto& kv : refs) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(kv.first.device);
        cudaFree(kv.second.state);
        cudaFree(kv.second.dims);
        cudaFree(kv.second.cap);
        cudaFree(kv.second.off);
        for (auto& pk : kv.second.packed) {
            cudaFree(pk.second.state);
            cudaFree(pk.second.cap);
            cudaFree(pk.second.off);
        }
        cudaSetDevice(cur);
    }
}

qc_status CircuitImpl::device_copy(DeviceCopy** out) {
    int d = 0;
    QC_CUDA(cudaGetDevice(&d));
    std::lock_guard<std::mutex> lk(mu);
    auto it = dev.find(d);
    if (it == dev.end()) {
        DeviceCopy dc;
        const size_t npre = pre.size() ? pre.size() : 1, nmps = mps.size() ? mps.size() : 1;
        const size_t nch = chan_kind.size() ? chan_kind.size() : 1;
        QC_CUDA(cudaMalloc(&dc.pre, npre * sizeof(PreOp)));
        QC_CUDA(cudaMalloc(&dc.mps, nmps * sizeof(MpsOp)));
        QC_CUDA(cudaMalloc(&dc.chan_kind, nch));
        if (!pre.empty()) QC_CUDA(cudaMemcpy(dc.pre, pre.data(), pre.size() * sizeof(PreOp), cudaMemcpyHostToDevice));
        if (!mps.empty()) QC_CUDA(cudaMemcpy(dc.mps, mps.data(), mps.size() * sizeof(MpsOp), cudaMemcpyHostToDevice));
        if (!chan_kind.empty()) QC_CUDA(cudaMemcpy(dc.chan_kind, chan_kind.data(), chan_kind.size(), cudaMemcpyHostToDevice));
        it = dev.emplace(d, dc).first;
    }
    *out = &it->second;
    return QC_OK;
}

}  // namespace qc

using namespace qc;

extern "C" const char* qc_last_error(void) { return g_last_error.c_str(); }

static bool parse_kind(const std::string& s, uint8_t& k, int& arity) {
    static const struct { const char* name; uint8_t kind; int ar; } tab[] = {
        {"H", K_H, 1}, {"S", K_S, 1}, {"SDG", K_SDG, 1}, {"X", K_X, 1}, {"Y", K_Y, 1}, {"Z", K_Z, 1},
        {"T", K_T, 1}, {"TDG", K_TDG, 1}, {"CX", K_CX, 2}, {"CZ", K_CZ, 2}, {"SWAP", K_SWAP, 2},
        {"M", K_M, 1}, {"R", K_R, 1}, {"DEP1", K_DEP1, 1}, {"DEP2", K_DEP2, 2}, {"XERR", K_XERR, 1}};
    for (const auto& e : tab)
        if (s == e.name) { k = e.kind; arity = e.ar; return true; }
    return false;
}

extern "C" qc_status qc_circuit_parse(const char* text, size_t len, qc_circuit** out) {
    if (!out || (!text && len)) return fail(QC_EINVAL, "null argument");
    *out = nullptr;
    std::unique_ptr<qc_circuit> cp(new qc_circuit());
    CircuitImpl& c = cp->impl;
    std::istringstream in(std::string(text ? text : "", len));
    std::string line;
    int lineno = 0;
    bool have_n = false;
    uint32_t nch = 0, nread = 0;
    while (std::getline(in, line)) {
        ++lineno;
        auto hash = line.find('#');
        if (hash != std::string::npos) line.resize(hash);
        std::istringstream ls(line);
        std::string name;
        if (!(ls >> name)) continue;
        for (auto& ch : name) ch = (char)toupper((unsigned char)ch);
        if (name == "QUBITS") {
            long n = -1;
            if (have_n || !(ls >> n) || n < 1 || n > 4095)
                return fail(QC_EINVAL, "line %d: bad QUBITS (1..4095, once)", lineno);
            c.n = (int)n;
            have_n = true;
            continue;
        }
        if (!have_n) return fail(QC_EINVAL, "line %d: QUBITS must come first", lineno);
        if (name == "TICK") continue;
        uint8_t kind;
        int arity;
        if (!parse_kind(name, kind, arity)) return fail(QC_EINVAL, "line %d: unknown instruction %s", lineno, name.c_str());
        long q[2] = {0, 0};
        for (int k = 0; k < arity; ++k)
            if (!(ls >> q[k]) || q[k] < 0 || q[k] >= c.n)
                return fail(QC_EINVAL, "line %d: %s needs %d qubit(s) in range", lineno, name.c_str(), arity);
        std::string extra;
        if (ls >> extra) return fail(QC_EINVAL, "line %d: trailing text", lineno);
        if (arity == 2 && q[0] == q[1]) return fail(QC_EINVAL, "line %d: %s on one qubit twice", lineno, name.c_str());
        Op op{kind, (int32_t)q[0], (int32_t)(arity == 2 ? q[1] : -1), 0};
        if (kind == K_DEP1 || kind == K_DEP2 || kind == K_XERR) {
            op.aux = nch++;
            c.chan_kind.push_back(kind == K_DEP1 ? 1 : kind == K_DEP2 ? 2 : 3);
        } else if (kind == K_M || kind == K_R) {
            op.aux = nread++;
            if (kind == K_M) ++c.n_meas; else ++c.n_resets;
        } else if (kind == K_T || kind == K_TDG) {
            ++c.n_t;
        }
        c.ops.push_back(op);
    }
    if (!have_n) return fail(QC_EINVAL, "empty circuit");
    c.n_readouts = nread;
    analyse(c);
    for (uint8_t d : c.decided) c.n_decided += d;
    compile_prescreen(c);
    compile_mps(c);
    *out = cp.release();
    return QC_OK;
}

extern "C" void qc_circuit_free(qc_circuit* circuit) { delete circuit; }

extern "C" qc_status qc_circuit_get_info(const qc_circuit* circuit, qc_circuit_info* out) {
    if (!circuit || !out) return fail(QC_EINVAL, "null argument");
    const CircuitImpl& c = circuit->impl;
    out->n_qubits = c.n;
    out->n_ops = (int64_t)c.ops.size();
    out->n_channels = (int64_t)c.chan_kind.size();
    out->n_measurements = c.n_meas;
    out->n_decided = c.n_decided;
    out->n_resets = c.n_resets;
    out->n_t = c.n_t;
    out->n_mps_updates = c.n_updates;
    out->n_product_swaps = c.n_pswaps;
    return QC_OK;
}

extern "C" qc_status qc_circuit_decided(const qc_circuit* circuit, uint8_t* flags) {
    if (!circuit || !flags) return fail(QC_EINVAL, "null argument");
    const auto& d = circuit->impl.decided;
    if (!d.empty()) memcpy(flags, d.data(), d.size());
    return QC_OK;
}
