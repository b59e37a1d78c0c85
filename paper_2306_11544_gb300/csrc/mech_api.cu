// C ABI of libmech (declared in include/mech.h): handle lifetime, device
// buffers, voxel grids, the per-step launch sequence, CUDA-graph replay and the
// caller-order read/write/checkpoint calls.  No allocation happens inside
// mech_step: every buffer is sized when the handle, its domain or its voxel
// side is set (the GPU form of the paper's first lesson, Sec. 4.3: no memory
// management inside the hot loop).
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mech.h"
#include "mech_internal.cuh"

using namespace mk;

namespace {

thread_local std::string g_err;
std::atomic<int> g_fault_alloc{0};  // host-armed: the next device allocation fails

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(expr)                                                                              \
    do {                                                                                            \
        cudaError_t e_ = (expr);                                                                    \
        if (e_ != cudaSuccess) return fail(MECH_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define MECH_TRY(expr)             \
    do {                           \
        int rc_ = (expr);          \
        if (rc_ != MECH_OK) return rc_; \
    } while (0)

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

int mk::record_error(int code, const std::string& msg) { return fail(code, msg); }

struct mech {
    int dev = 0;
    int sms = 152;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int mode = kMixedFP64Pos;
    int64_t n = 0;
    int32_t nrep = 0;
    uint32_t npad = 0;
    std::vector<int64_t> counts, cbase;
    std::vector<std::array<double, 3>> dom_lo, dom_hi;
    std::vector<bool> dom_auto;
    std::vector<double> maxabs;  // per replicate, for the default domain
    double maxR = 0.0;
    double A = 0.0, voxel_user = 0.0, voxel_int = 0.0, dt = 0.0;
    bool params_set = false;
    bool grid_dirty = true;
    // grids
    std::vector<GridDev> grids;
    uint32_t V = 0, Vpad = 0;
    GridDev* d_grids = nullptr;
    size_t grid_cap = 0;
    // voxel tiles
    int ltx = 2, lty = 2, ltz = 2;
    bool use_tiles = true;
    // velocity variants
    int32_t max_type = -1;         // largest cell type created or added so far
    int32_t ntypes = 0;            // > 0: affinity table in use
    float* d_aff_f = nullptr;      // 16 x 16 affinity tables (FP32, FP64)
    double* d_aff_d = nullptr;
    int32_t walls = 0;
    double c_wall = 0.0;
    int tile_kernel = kTileKernelCTA;
    uint32_t dense_min = 12;
    uint32_t NT = 0;
    size_t tcap = 0;
    uint32_t* d_tcount[2] = {nullptr, nullptr};
    uint8_t* d_tdense = nullptr;
    uint32_t* d_tlist = nullptr;
    uint32_t* d_ndense = nullptr;
    uint2* d_slist = nullptr;
    uint32_t* d_nsparse = nullptr;
    unsigned long long* d_stats = nullptr;  // mech_pair_stats counters
    // state
    StateBuf st[2] = {};
    int cur = 0;
    double* d_R64 = nullptr;
    double* d_ccr64 = nullptr;
    double* d_cca64 = nullptr;
    // binning scratch
    uint32_t* d_key = nullptr;
    uint32_t* d_vkey_s = nullptr;
    uint32_t* d_perm = nullptr;
    unsigned long long* d_tmp = nullptr;
    uint32_t* d_count[2] = {nullptr, nullptr};
    uint32_t* d_start = nullptr;
    uint32_t* d_bsum = nullptr;
    uint32_t* d_bcount[2] = {nullptr, nullptr};  // cells per scan block, this step and the next
    uint32_t* d_occ = nullptr;
    size_t vcap = 0;  // capacity (entries) of count/start
    double* d_io = nullptr;  // 6n doubles of staging
    // mech_remove_cells scratch (allocated at first use): alive bytes, scan
    // flags, two prefix arrays and the scan's block sums, for ccap cells
    uint8_t* d_alive = nullptr;
    uint32_t* d_cflags = nullptr;
    uint32_t* d_cpref[2] = {nullptr, nullptr};
    uint32_t* d_cbsum = nullptr;
    size_t ccap = 0;
    uint32_t* d_shift = nullptr;  // mech_add_cells_batch: per-replicate shift
    size_t shift_cap = 0;
    float* d_vout_f = nullptr;
    double* d_vout_d = nullptr;
    bool vout_valid = false;
    uint32_t* d_err = nullptr;
    bool keys_valid = false;
    int64_t step = 0;
    int force_block = 256;
    uint32_t fault = 0;            // host-armed fault injection (kFault* bits)
    bool poisoned = false;         // a device error left the state inconsistent
    int force_grid = 0;
    int tile_grid = 0;
    int elem_grid = 0;
    // graphs: one per starting parity of `cur`
    int graph_steps = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    size_t dev_bytes = 0;
    std::vector<void*> allocs;
    // per-phase profiling: kProfPhases + 1 events per recorded step
    static constexpr int kProfPhases = 6;
    static constexpr int kProfCap = 4096;
    bool profiling = false;
    std::vector<cudaEvent_t> prof_ev;
    int prof_steps = 0;

    ~mech() {
        for (cudaEvent_t e : prof_ev) cudaEventDestroy(e);
        for (int p = 0; p < 2; ++p)
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
        for (void* p : allocs) cudaFree(p);
        if (own_stream) cudaStreamDestroy(own_stream);
    }

    template <typename T>
    int alloc(T** p, size_t count) {
        *p = nullptr;
        size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        void* q = nullptr;
        int armed = 1;
        if (g_fault_alloc.compare_exchange_strong(armed, 0))
            return fail(MECH_E_OOM, "injected allocation failure (mech_debug_inject)");
        cudaError_t e = cudaMalloc(&q, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(MECH_E_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                        cudaGetErrorString(e));
        }
        allocs.push_back(q);
        dev_bytes += bytes;
        *p = static_cast<T*>(q);
        // scratch starts at zero: indices read from it are always in range
        if (cudaMemset(q, 0, bytes) != cudaSuccess)
            return fail(MECH_E_CUDA, "cudaMemset of a new buffer failed");
        return MECH_OK;
    }

    void free_ptr(void* p, size_t bytes) {
        if (!p) return;
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) allocs.erase(it);
        cudaFree(p);
        dev_bytes -= bytes;
    }

    void invalidate_graphs() {
        for (int p = 0; p < 2; ++p)
            if (gexec[p]) {
                cudaGraphExecDestroy(gexec[p]);
                gexec[p] = nullptr;
            }
    }

    StepArgs args(int a_idx, int integrate) const {
        StepArgs a{};
        a.mode = mode;
        a.n = (uint32_t)n;
        a.npad = npad;
        a.nrep = nrep;
        a.grids = d_grids;
        a.A = st[a_idx];
        a.B = st[a_idx ^ 1];
        a.key = d_key;
        a.vkey_s = d_vkey_s;
        a.perm = d_perm;
        a.tmp = d_tmp;
        a.count_cur = d_count[a_idx];
        a.count_nxt = d_count[a_idx ^ 1];
        a.bcount_cur = d_bcount[a_idx];
        a.bcount_nxt = d_bcount[a_idx ^ 1];
        a.start = d_start;
        a.occ = d_occ;
        a.R64 = d_R64;
        a.ccr64 = d_ccr64;
        a.cca64 = d_cca64;
        a.A_f = (float)A;
        a.A2m1_f = (float)(A * A - 1.0);
        a.dt_f = (float)dt;
        a.A_d = A;
        a.dt_d = dt;
        a.integrate = integrate;
        a.vout_f = d_vout_f;
        a.vout_d = d_vout_d;
        a.err = d_err;
        a.ltx = ltx;
        a.lty = lty;
        a.ltz = ltz;
        a.use_tiles = use_tiles ? 1 : 0;
        a.ntypes = ntypes;
        a.aff_f = d_aff_f;
        a.aff_d = d_aff_d;
        a.walls = walls;
        a.c_wall = c_wall;
        a.tile_kernel = tile_kernel;
        a.ntiles = NT;
        a.dense_min = dense_min;
        a.tcount_cur = d_tcount[a_idx];
        a.tcount_nxt = d_tcount[a_idx ^ 1];
        a.tdense = d_tdense;
        a.tlist = d_tlist;
        a.ndense = d_ndense;
        a.slist = d_slist;
        a.nsparse = d_nsparse;
        a.cut_eps = (float)(2e-5 * A * maxR);
        a.fault = fault;
        a.wait_ns = (fault & kFaultTileWait) ? 1000000ull : 2000000000ull;  // 1 ms armed, 2 s otherwise
        return a;
    }
};

namespace {

int check_handle(mech_t* h) {
    if (!h) return fail(MECH_E_ARG, "null handle");
    return MECH_OK;
}

double voxel_of(const mech_t* h) { return h->voxel_int > 0.0 ? h->voxel_int : h->voxel_user; }

// Build the per-replicate grids for the current voxel side and domains, and
// size the voxel arrays.  Called outside the step loop only.
int build_grids(mech_t* h) {
    const double vx = voxel_of(h);
    std::vector<GridDev> g(h->nrep);
    uint64_t vsum = 0, tsum = 0;
    for (int r = 0; r < h->nrep; ++r) {
        double lo[3], hi[3];
        if (h->dom_auto[r]) {
            double half = std::max(1.5 * h->maxabs[r], 0.5 * vx);
            for (int d = 0; d < 3; ++d) { lo[d] = -half; hi[d] = half; }
        } else {
            for (int d = 0; d < 3; ++d) { lo[d] = h->dom_lo[r][d]; hi[d] = h->dom_hi[r][d]; }
        }
        GridDev& G = g[r];
        for (int d = 0; d < 3; ++d) {
            double nd = std::ceil((hi[d] - lo[d]) / vx);
            if (!(nd >= 1.0)) nd = 1.0;
            if (nd > (double)(1 << 21)) return fail(MECH_E_OOM, "grid has more than 2^21 voxels along an axis");
            G.n[d] = (int32_t)nd;
            G.lo[d] = lo[d];
            G.lo_f[d] = (float)lo[d];
        }
        for (int d = 0; d < 3; ++d) {
            G.whi[d] = hi[d];
            G.whi_f[d] = (float)hi[d];
        }
        G.h = vx;
        G.inv_h = 1.0 / vx;
        G.h_f = (float)vx;
        G.inv_h_f = (float)(1.0 / vx);
        G.vbase = (uint32_t)vsum;
        G.cbase = (uint32_t)h->cbase[r];
        G.ncell = (uint32_t)h->counts[r];
        vsum += (uint64_t)G.n[0] * (uint64_t)G.n[1] * (uint64_t)G.n[2];
        const int lt[3] = {h->ltx, h->lty, h->ltz};
        for (int d = 0; d < 3; ++d) G.nt[d] = (G.n[d] + (1 << lt[d]) - 1) >> lt[d];
        // record origin: the grid centre; hi grid q: 2^23 q covers twice the
        // largest half-extent, so cells up to one half-extent outside the grid
        // stay on it
        double half = 0.0;
        for (int d = 0; d < 3; ++d) {
            G.oc[d] = lo[d] + 0.5 * (double)G.n[d] * vx;
            G.oc_hi[d] = (float)G.oc[d];
            G.oc_lo[d] = (float)(G.oc[d] - (double)G.oc_hi[d]);
            half = std::max(half, 0.5 * (double)G.n[d] * vx);
        }
        const int k = 23 - (int)std::ceil(std::log2(2.0 * half));
        G.q = (float)std::ldexp(1.0, -k);
        G.inv_q = (float)std::ldexp(1.0, k);
        G.qs = (float)std::ldexp(1.0, -k - 15);
        G.qm = 2.0f * G.q;
        G.qexp = -k;
        G.qf24 = (float)std::ldexp(1.0, -k - 24);
        G.fix_ok = 1;
        for (int d = 0; d < 3; ++d) {
            const double f = std::ldexp(G.oc[d], k + 24);
            if (!(std::fabs(f) < std::ldexp(1.0, 61))) G.fix_ok = 0;
            G.oc_fix[d] = G.fix_ok ? std::llround(f) : 0;
        }
        G.tbase = (uint32_t)tsum;
        tsum += (uint64_t)G.nt[0] * (uint64_t)G.nt[1] * (uint64_t)G.nt[2];
        if (vsum > (uint64_t)0x7FFFFFFF - 2 * (uint64_t)kScanTile)
            return fail(MECH_E_OOM, "voxel grids exceed 2^31 voxels; enlarge the voxel or shrink the domain");
    }
    const uint32_t V = (uint32_t)vsum;
    const size_t Vpad = ((size_t)V + 1 + kScanTile - 1) / kScanTile * kScanTile;
    // (re)allocate voxel arrays if they grew
    if (Vpad > h->vcap) {
        for (int p = 0; p < 2; ++p) h->free_ptr(h->d_count[p], h->vcap * 4);
        h->free_ptr(h->d_start, h->vcap * 4);
        h->free_ptr(h->d_bsum, h->vcap / kScanTile * 4);
        for (int p = 0; p < 2; ++p) h->free_ptr(h->d_bcount[p], h->vcap / kScanTile * 4);
        h->free_ptr(h->d_occ, (h->vcap / 32 + 1) * 4);
        h->d_count[0] = h->d_count[1] = nullptr;
        h->d_start = nullptr;
        h->d_bsum = nullptr;
        h->d_bcount[0] = h->d_bcount[1] = nullptr;
        h->d_occ = nullptr;
        h->vcap = 0;
        MECH_TRY(h->alloc(&h->d_count[0], Vpad));
        MECH_TRY(h->alloc(&h->d_count[1], Vpad));
        MECH_TRY(h->alloc(&h->d_start, Vpad));
        MECH_TRY(h->alloc(&h->d_bsum, Vpad / kScanTile));
        MECH_TRY(h->alloc(&h->d_bcount[0], Vpad / kScanTile));
        MECH_TRY(h->alloc(&h->d_bcount[1], Vpad / kScanTile));
        MECH_TRY(h->alloc(&h->d_occ, Vpad / 32 + 1));
        h->vcap = Vpad;
    }
    const uint32_t NT = (uint32_t)tsum;
    if ((size_t)NT + 1 > h->tcap) {
        for (int p = 0; p < 2; ++p) h->free_ptr(h->d_tcount[p], h->tcap * 4);
        h->free_ptr(h->d_tdense, h->tcap);
        h->free_ptr(h->d_tlist, h->tcap * 4);
        h->d_tcount[0] = h->d_tcount[1] = nullptr;
        h->d_tdense = nullptr;
        h->d_tlist = nullptr;
        h->tcap = 0;
        const size_t cap = (size_t)NT + 1;
        MECH_TRY(h->alloc(&h->d_tcount[0], cap));
        MECH_TRY(h->alloc(&h->d_tcount[1], cap));
        MECH_TRY(h->alloc(&h->d_tdense, cap));
        MECH_TRY(h->alloc(&h->d_tlist, cap));
        h->tcap = cap;
    }
    if ((size_t)h->nrep > h->grid_cap) {
        h->free_ptr(h->d_grids, h->grid_cap * sizeof(GridDev));
        h->d_grids = nullptr;
        MECH_TRY(h->alloc(&h->d_grids, (size_t)h->nrep));
        h->grid_cap = h->nrep;
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_grids, g.data(), g.size() * sizeof(GridDev), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_count[0], Vpad, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_count[1], Vpad, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_bcount[0], Vpad / kScanTile, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_bcount[1], Vpad / kScanTile, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_occ, Vpad / 32 + 1, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_tcount[0], NT, h->stream));
    CUDA_TRY(launch_zero_u32(h->d_tcount[1], NT, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));  // host vectors die here
    h->grids = g;
    h->NT = NT;
    h->V = V;
    h->Vpad = (uint32_t)Vpad;
    h->grid_dirty = false;
    h->keys_valid = false;
    h->invalidate_graphs();
    return MECH_OK;
}

int ready(mech_t* h) {
    MECH_TRY(check_handle(h));
    if (!h->params_set) return fail(MECH_E_STATE, "mech_set_params must be called before stepping");
    if (h->grid_dirty) MECH_TRY(build_grids(h));
    return MECH_OK;
}

int ensure_keys(mech_t* h) {
    if (h->keys_valid) return MECH_OK;
    StepArgs a = h->args(h->cur, 1);
    for (int p = 0; p < 2; ++p) {  // this step's histograms are rebuilt; the next step's start from zero
        CUDA_TRY(launch_zero_u32(h->d_count[p], h->Vpad, h->stream));
        CUDA_TRY(launch_zero_u32(h->d_bcount[p], h->Vpad / kScanTile, h->stream));
        CUDA_TRY(launch_zero_u32(h->d_tcount[p], h->NT, h->stream));
    }
    CUDA_TRY(launch_keys(a, h->elem_grid, h->Vpad, h->stream));
    h->keys_valid = true;
    return MECH_OK;
}

// Enqueue one step from st[cur]; flips cur.  Needs valid keys.
int enqueue_step(mech_t* h, int integrate, bool profile = false) {
    StepArgs a = h->args(h->cur, integrate);
    cudaEvent_t* ev = nullptr;
    if (profile && h->prof_steps < mech::kProfCap) ev = &h->prof_ev[(size_t)h->prof_steps * (mech::kProfPhases + 1)];
    if (ev) CUDA_TRY(cudaEventRecord(ev[0], h->stream));
    // the scan starts from the histogram's block sums (counted by the previous
    // step's force epilogue, or summed by the reduce pass after k_keys) and
    // clears the next step's block sums
    CUDA_TRY(launch_scan_blocks(a.count_cur, h->Vpad, a.bcount_cur, a.bcount_nxt, h->d_start, h->d_ndense,
                                h->d_occ, h->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[1], h->stream));
    CUDA_TRY(launch_scatter(a, h->elem_grid, h->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[2], h->stream));
    CUDA_TRY(launch_canon(a, h->elem_grid, h->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[3], h->stream));
    CUDA_TRY(launch_tile_classify(a, h->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[4], h->stream));
    CUDA_TRY(launch_force_tiles(a, h->tile_grid, h->stream));
    if (ev) CUDA_TRY(cudaEventRecord(ev[5], h->stream));
    CUDA_TRY(launch_sparse_list(a, h->elem_grid, h->stream));
    CUDA_TRY(launch_force_cells(a, h->force_grid, h->force_block, h->stream));
    if (ev) {
        CUDA_TRY(cudaEventRecord(ev[6], h->stream));
        ++h->prof_steps;
    }
    h->cur ^= 1;
    return MECH_OK;
}

int capture_graph(mech_t* h) {
    const int parity = h->cur;
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    int rc = MECH_OK;
    for (int s = 0; s < h->graph_steps && rc == MECH_OK; ++s) rc = enqueue_step(h, 1);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    h->cur = parity;  // capture only recorded the launches
    if (rc != MECH_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return fail(MECH_E_CUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec[parity], graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MECH_E_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    return MECH_OK;
}

int check_err_flag(mech_t* h) {
    uint32_t e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, h->d_err, sizeof(uint32_t), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (e) {
        cudaMemsetAsync(h->d_err, 0, sizeof(uint32_t), h->stream);
        cudaStreamSynchronize(h->stream);
        h->poisoned = true;
        if (e & kErrTimeout)
            return fail(MECH_E_TIMEOUT, "a bounded wait in the tile kernel gave up (TMA copy did not complete)");
        return fail(MECH_E_DEVICE_FLAG, std::string("device error flag raised: ") +
                                            ((e & kErrNonFinite) ? "non-finite position or velocity " : "") +
                                            ((e & kErrIndex) ? "index out of range" : ""));
    }
    return MECH_OK;
}

int validate_cells(int64_t n, const double* xyz, const double* R, const double* ccr, const double* cca) {
    if (n < 0) return fail(MECH_E_ARG, "negative cell count");
    if (n > 0 && (!xyz || !R || !ccr || !cca)) return fail(MECH_E_ARG, "null input array");
    if (n >= (int64_t)0x7FFFFFFF) return fail(MECH_E_ARG, "more than 2^31-1 cells");
    if (!finite_all(xyz, 3 * (size_t)n) || !finite_all(R, n) || !finite_all(ccr, n) || !finite_all(cca, n))
        return fail(MECH_E_NONFINITE, "non-finite value in the cell arrays");
    for (int64_t i = 0; i < n; ++i) {
        if (!(R[i] > 0.0)) return fail(MECH_E_ARG, "radius must be > 0 (cell " + std::to_string(i) + ")");
        if (ccr[i] < 0.0 || cca[i] < 0.0)
            return fail(MECH_E_ARG, "ccr and cca must be >= 0 (cell " + std::to_string(i) + ")");
    }
    return MECH_OK;
}

// Per-cell device buffers of a capacity of np cells (the SoA component
// stride): both state buffers, FP64 parameters in caller order, binning
// scratch, staging and velocities-only outputs.
struct CellBuffers {
    StateBuf st[2] = {};
    double* R64 = nullptr;
    double* ccr64 = nullptr;
    double* cca64 = nullptr;
    uint32_t* key = nullptr;
    uint2* slist = nullptr;
    uint32_t* vkey_s = nullptr;
    uint32_t* perm = nullptr;
    unsigned long long* tmp = nullptr;
    double* io = nullptr;
    float* vout_f = nullptr;
    double* vout_d = nullptr;
};

int alloc_cell_buffers(mech_t* h, size_t np, CellBuffers& b) {
    b = CellBuffers{};
    int rc = MECH_OK;
    for (int s = 0; s < 2 && rc == MECH_OK; ++s) {
        StateBuf& x = b.st[s];
        rc = h->alloc(&x.pos64, 3 * np);
        if (rc == MECH_OK) rc = h->alloc(&x.posf, 3 * np);
        if (rc == MECH_OK) rc = h->alloc(&x.comp, 3 * np);
        if (rc == MECH_OK) rc = h->alloc(&x.vp64, 3 * np);
        if (rc == MECH_OK) rc = h->alloc(&x.vpf, 3 * np);
        if (rc == MECH_OK) rc = h->alloc(&x.id, np);
        if (rc == MECH_OK) rc = h->alloc(&x.rec, 2 * np);
    }
    if (rc == MECH_OK) rc = h->alloc(&b.R64, np);
    if (rc == MECH_OK) rc = h->alloc(&b.ccr64, np);
    if (rc == MECH_OK) rc = h->alloc(&b.cca64, np);
    if (rc == MECH_OK) rc = h->alloc(&b.key, np);
    if (rc == MECH_OK) rc = h->alloc(&b.slist, np);
    if (rc == MECH_OK) rc = h->alloc(&b.vkey_s, np);
    if (rc == MECH_OK) rc = h->alloc(&b.perm, np);
    if (rc == MECH_OK) rc = h->alloc(&b.tmp, np);
    if (rc == MECH_OK) rc = h->alloc(&b.io, 6 * np);
    if (rc == MECH_OK) rc = h->alloc(&b.vout_f, 3 * np);
    if (rc == MECH_OK) rc = h->alloc(&b.vout_d, 3 * np);
    return rc;
}

// Frees what alloc_cell_buffers allocated (null pointers are skipped).
void free_cell_buffers(mech_t* h, const CellBuffers& b, size_t np) {
    for (int s = 0; s < 2; ++s) {
        const StateBuf& x = b.st[s];
        h->free_ptr(x.pos64, 3 * np * 8);
        h->free_ptr(x.posf, 3 * np * 4);
        h->free_ptr(x.comp, 3 * np * 4);
        h->free_ptr(x.vp64, 3 * np * 8);
        h->free_ptr(x.vpf, 3 * np * 4);
        h->free_ptr(x.id, np * 4);
        h->free_ptr(x.rec, 2 * np * sizeof(float4));
    }
    h->free_ptr(b.R64, np * 8);
    h->free_ptr(b.ccr64, np * 8);
    h->free_ptr(b.cca64, np * 8);
    h->free_ptr(b.key, np * 4);
    h->free_ptr(b.slist, np * sizeof(uint2));
    h->free_ptr(b.vkey_s, np * 4);
    h->free_ptr(b.perm, np * 4);
    h->free_ptr(b.tmp, np * 8);
    h->free_ptr(b.io, 6 * np * 8);
    h->free_ptr(b.vout_f, 3 * np * 4);
    h->free_ptr(b.vout_d, 3 * np * 8);
}

CellBuffers cell_buffers_of(const mech_t* h) {
    CellBuffers b;
    b.st[0] = h->st[0];
    b.st[1] = h->st[1];
    b.R64 = h->d_R64;
    b.ccr64 = h->d_ccr64;
    b.cca64 = h->d_cca64;
    b.key = h->d_key;
    b.slist = h->d_slist;
    b.vkey_s = h->d_vkey_s;
    b.perm = h->d_perm;
    b.tmp = h->d_tmp;
    b.io = h->d_io;
    b.vout_f = h->d_vout_f;
    b.vout_d = h->d_vout_d;
    return b;
}

void set_cell_buffers(mech_t* h, const CellBuffers& b) {
    h->st[0] = b.st[0];
    h->st[1] = b.st[1];
    h->d_R64 = b.R64;
    h->d_ccr64 = b.ccr64;
    h->d_cca64 = b.cca64;
    h->d_key = b.key;
    h->d_slist = b.slist;
    h->d_vkey_s = b.vkey_s;
    h->d_perm = b.perm;
    h->d_tmp = b.tmp;
    h->d_io = b.io;
    h->d_vout_f = b.vout_f;
    h->d_vout_d = b.vout_d;
}

// Moves the per-cell buffers to a capacity of cap2 >= n cells: the current
// state (SoA rows re-strided), ids, records and FP64 parameters are copied;
// the other state buffer and the scratch need no copy (keys are recomputed).
int grow_capacity(mech_t* h, size_t cap2) {
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    const size_t np = h->npad, n = (size_t)h->n;
    const CellBuffers old = cell_buffers_of(h);
    CellBuffers nb;
    const int rc = alloc_cell_buffers(h, cap2, nb);
    if (rc != MECH_OK) {
        free_cell_buffers(h, nb, cap2);
        return rc;
    }
    if (n > 0) {
        const StateBuf& so = old.st[h->cur];
        const StateBuf& sn = nb.st[h->cur];
        auto rows3 = [&](void* dst, const void* src, size_t es) {
            return cudaMemcpy2DAsync(dst, cap2 * es, src, np * es, n * es, 3, cudaMemcpyDeviceToDevice, h->stream);
        };
        auto flat = [&](void* dst, const void* src, size_t bytes) {
            return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToDevice, h->stream);
        };
        cudaError_t e = rows3(sn.pos64, so.pos64, 8);
        if (e == cudaSuccess) e = rows3(sn.posf, so.posf, 4);
        if (e == cudaSuccess) e = rows3(sn.comp, so.comp, 4);
        if (e == cudaSuccess) e = rows3(sn.vp64, so.vp64, 8);
        if (e == cudaSuccess) e = rows3(sn.vpf, so.vpf, 4);
        if (e == cudaSuccess) e = flat(sn.id, so.id, n * 4);
        if (e == cudaSuccess) e = flat(sn.rec, so.rec, 2 * n * sizeof(float4));
        if (e == cudaSuccess) e = flat(nb.R64, old.R64, n * 8);
        if (e == cudaSuccess) e = flat(nb.ccr64, old.ccr64, n * 8);
        if (e == cudaSuccess) e = flat(nb.cca64, old.cca64, n * 8);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) {
            free_cell_buffers(h, nb, cap2);
            return fail(MECH_E_CUDA, std::string("capacity growth: ") + cudaGetErrorString(e));
        }
    }
    set_cell_buffers(h, nb);
    free_cell_buffers(h, old, np);
    h->npad = (uint32_t)cap2;
    h->keys_valid = false;
    h->vout_valid = false;
    h->invalidate_graphs();
    return MECH_OK;
}

// Bookkeeping after the cell counts changed: per-replicate counts and first
// cells, the grid descriptors' cell ranges (the device copy too, when the
// grids are built), launch sizes; keys, velocities-only output and graphs
// are invalid.
int set_cell_counts(mech_t* h, const std::vector<int64_t>& counts) {
    h->counts = counts;
    int64_t run = 0;
    for (int r = 0; r < h->nrep; ++r) {
        h->cbase[r] = run;
        run += counts[r];
    }
    h->n = run;
    h->elem_grid = (int)std::min<int64_t>(std::max<int64_t>(h->sms * 8, (run + 1023) / 1024), 1 << 20);
    h->keys_valid = false;
    h->vout_valid = false;
    h->invalidate_graphs();
    if (!h->grid_dirty && (int)h->grids.size() == h->nrep && h->d_grids) {
        for (int r = 0; r < h->nrep; ++r) {
            h->grids[r].cbase = (uint32_t)h->cbase[r];
            h->grids[r].ncell = (uint32_t)h->counts[r];
        }
        CUDA_TRY(cudaMemcpyAsync(h->d_grids, h->grids.data(), h->grids.size() * sizeof(GridDev),
                                 cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host copy may change again
    }
    return MECH_OK;
}

// Cell types must lie in [0, 16) (they travel in 4 bits of the force
// record); returns the largest one (-1 for none).
int check_types(int64_t n, const int32_t* type, int32_t& max_type) {
    max_type = -1;
    if (!type) {
        if (n > 0) max_type = 0;
        return MECH_OK;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (type[i] < 0 || type[i] >= kMaxTypes) return fail(MECH_E_ARG, "cell types must lie in [0, 16)");
        max_type = std::max(max_type, type[i]);
    }
    return MECH_OK;
}

int create_impl(mech_t** out, int32_t nrep, const int64_t* counts, const double* xyz, const double* R,
                const double* ccr, const double* cca, const int32_t* type) {
    int64_t n = 0;
    for (int r = 0; r < nrep; ++r) {
        if (counts[r] < 0) return fail(MECH_E_ARG, "negative replicate count");
        n += counts[r];
    }
    MECH_TRY(validate_cells(n, xyz, R, ccr, cca));
    int32_t max_type = -1;
    MECH_TRY(check_types(n, type, max_type));
    mech_t* h = new (std::nothrow) mech_t();
    if (!h) return fail(MECH_E_OOM, "host allocation failed");
    auto bail = [&](int rc) {
        delete h;
        return rc;
    };
    cudaError_t e = cudaGetDevice(&h->dev);
    if (e != cudaSuccess) return bail(fail(MECH_E_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e)));
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, h->dev);
    if (e != cudaSuccess) return bail(fail(MECH_E_CUDA, std::string("cudaGetDeviceProperties: ") + cudaGetErrorString(e)));
    h->sms = prop.multiProcessorCount;
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(fail(MECH_E_CUDA, std::string("cudaStreamCreate: ") + cudaGetErrorString(e)));
    h->stream = h->own_stream;
    h->n = n;
    h->nrep = nrep;
    h->max_type = max_type;
    h->npad = (uint32_t)((n + 63) / 64 * 64);
    if (h->npad == 0) h->npad = 64;
    h->counts.assign(counts, counts + nrep);
    h->cbase.resize(nrep);
    int64_t run = 0;
    for (int r = 0; r < nrep; ++r) { h->cbase[r] = run; run += counts[r]; }
    h->dom_lo.assign(nrep, {0, 0, 0});
    h->dom_hi.assign(nrep, {0, 0, 0});
    h->dom_auto.assign(nrep, true);
    h->maxabs.assign(nrep, 0.0);
    for (int r = 0; r < nrep; ++r)
        for (int64_t i = h->cbase[r]; i < h->cbase[r] + counts[r]; ++i)
            for (int d = 0; d < 3; ++d) h->maxabs[r] = std::max(h->maxabs[r], std::fabs(xyz[3 * i + d]));
    for (int64_t i = 0; i < n; ++i) h->maxR = std::max(h->maxR, R[i]);

    const size_t np = h->npad;
    CellBuffers cb;
    int rc = alloc_cell_buffers(h, np, cb);
    set_cell_buffers(h, cb);
    if (rc == MECH_OK) rc = h->alloc(&h->d_nsparse, 2);
    if (rc == MECH_OK) rc = h->alloc(&h->d_stats, 2);
    if (rc == MECH_OK) rc = h->alloc(&h->d_err, 1);
    if (rc == MECH_OK) rc = h->alloc(&h->d_ndense, 1);
    if (rc != MECH_OK) return bail(rc);

    // caller order = initial state order; parameters and ids
    std::vector<uint32_t> ids(n);
    std::vector<float4> rec(2 * n);
    for (int64_t i = 0; i < n; ++i) {
        ids[i] = (uint32_t)i;
        // radius as FP32 + 12-bit residual in units of ulp(R) / 2^11 and the
        // type (upper half of the second float4); position residual fields
        // start at zero (0x8000)
        const float Rf = (float)R[i];
        const uint32_t wzr = 0x8000u | radius_type_bits(R[i], Rf, type ? (uint32_t)type[i] : 0u);
        float wzf, wxyf;
        const uint32_t wxy = 0x80008000u;
        std::memcpy(&wzf, &wzr, 4);
        std::memcpy(&wxyf, &wxy, 4);
        rec[2 * i] = make_float4(0.f, 0.f, 0.f, Rf);
        rec[2 * i + 1] = make_float4((float)std::sqrt(ccr[i]), (float)std::sqrt(cca[i]), wxyf, wzf);
    }
    cudaStream_t s = h->stream;
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    cudaError_t ce = cudaSuccess;
    if (ce == cudaSuccess) ce = up(h->st[0].id, ids.data(), n * 4);
    if (ce == cudaSuccess) ce = up(h->st[0].rec, rec.data(), 2 * n * sizeof(float4));
    if (ce == cudaSuccess) ce = up(h->d_R64, R, n * 8);
    if (ce == cudaSuccess) ce = up(h->d_ccr64, ccr, n * 8);
    if (ce == cudaSuccess) ce = up(h->d_cca64, cca, n * 8);
    if (ce == cudaSuccess) ce = up(h->d_io, xyz, 3 * n * 8);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->d_err, 0, 4, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(h->d_ndense, 0, 4, s);
    if (ce != cudaSuccess) return bail(fail(MECH_E_CUDA, std::string("upload: ") + cudaGetErrorString(ce)));
    StepArgs a = h->args(0, 1);
    ce = launch_load_pos(a, h->st[0], h->d_io, 0, nullptr, s);
    if (ce == cudaSuccess) ce = launch_load_vprev(a, h->st[0], nullptr, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return bail(fail(MECH_E_CUDA, std::string("initial load: ") + cudaGetErrorString(ce)));
    // element-wise kernels (binning): about four cells per thread, so that many
    // gathers are in flight (measured better than a grid-stride loop over a
    // few CTAs per SM)
    h->elem_grid = (int)std::min<int64_t>(std::max<int64_t>(h->sms * 8, (n + 1023) / 1024), 1 << 20);
    h->force_grid = h->sms * force_max_blocks_per_sm(h->mode, h->force_block);
    h->tile_grid = tile_kernel_grid(h->args(0, 1), h->sms);
    *out = h;
    return MECH_OK;
}

// positions (value) and previous velocities of st[cur] -> device io buffers, caller order
int stage_out(mech_t* h) {
    StepArgs a = h->args(h->cur, 1);
    const StateBuf& s = h->st[h->cur];
    CUDA_TRY(launch_unpermute_pos(a, s, h->d_io, h->d_io + 3 * (size_t)h->npad, h->d_tmp,
                                 8 * (size_t)h->npad, h->stream));
    if (h->mode == kFP64)
        CUDA_TRY(launch_unpermute_vel(a, s, nullptr, s.vp64, h->d_io + 3 * (size_t)h->npad, h->stream));
    else
        CUDA_TRY(launch_unpermute_vel(a, s, s.vpf, nullptr, h->d_io + 3 * (size_t)h->npad, h->stream));
    return MECH_OK;
}

}  // namespace

extern "C" {

const char* mech_last_error(void) { return g_err.c_str(); }

int mech_version(void) { return 100; }

int mech_create(mech_t** h, int64_t n, const double* xyz, const double* R, const double* ccr, const double* cca,
                const int32_t* type) {
    if (!h) return fail(MECH_E_ARG, "null output handle pointer");
    *h = nullptr;
    return create_impl(h, 1, &n, xyz, R, ccr, cca, type);
}

int mech_create_batch(mech_t** h, int32_t n_rep, const int64_t* counts, const double* xyz, const double* R,
                      const double* ccr, const double* cca, const int32_t* type) {
    if (!h) return fail(MECH_E_ARG, "null output handle pointer");
    *h = nullptr;
    if (n_rep < 1 || !counts) return fail(MECH_E_ARG, "n_rep must be >= 1 with a counts array");
    return create_impl(h, n_rep, counts, xyz, R, ccr, cca, type);
}

int mech_set_params(mech_t* h, double A, double voxel_size, double dt) {
    MECH_TRY(check_handle(h));
    if (!std::isfinite(A) || !std::isfinite(voxel_size) || !std::isfinite(dt))
        return fail(MECH_E_NONFINITE, "non-finite parameter");
    if (!(A >= 1.0)) return fail(MECH_E_ARG, "adhesion factor A must be >= 1");
    if (!(dt > 0.0)) return fail(MECH_E_ARG, "dt must be > 0");
    if (!(voxel_size > 0.0)) return fail(MECH_E_ARG, "voxel_size must be > 0");
    if (voxel_size < 2.0 * A * h->maxR)
        return fail(MECH_E_VOXEL_TOO_SMALL, "voxel_size must be >= 2 A max R = " + std::to_string(2.0 * A * h->maxR));
    if (h->voxel_int > 0.0 && h->voxel_int < 2.0 * A * h->maxR * (1.0 + 1e-6)) h->voxel_int = 0.0;
    if (voxel_size != h->voxel_user || voxel_of(h) != voxel_size) h->grid_dirty = true;
    h->A = A;
    h->voxel_user = voxel_size;
    h->dt = dt;
    h->params_set = true;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_set_domain(mech_t* h, int32_t rep, const double lo[3], const double hi[3]) {
    MECH_TRY(check_handle(h));
    if (!lo || !hi) return fail(MECH_E_ARG, "null domain corner");
    if (rep < -1 || rep >= h->nrep) return fail(MECH_E_ARG, "replicate index out of range");
    for (int d = 0; d < 3; ++d) {
        if (!std::isfinite(lo[d]) || !std::isfinite(hi[d])) return fail(MECH_E_NONFINITE, "non-finite domain");
        if (!(hi[d] > lo[d])) return fail(MECH_E_ARG, "domain needs lo < hi on every axis");
    }
    for (int r = (rep < 0 ? 0 : rep); r < (rep < 0 ? h->nrep : rep + 1); ++r) {
        h->dom_auto[r] = false;
        for (int d = 0; d < 3; ++d) { h->dom_lo[r][d] = lo[d]; h->dom_hi[r][d] = hi[d]; }
    }
    h->grid_dirty = true;
    if (h->params_set) return build_grids(h);
    return MECH_OK;
}

int mech_set_internal_voxel(mech_t* h, double voxel) {
    MECH_TRY(check_handle(h));
    if (!std::isfinite(voxel)) return fail(MECH_E_NONFINITE, "non-finite voxel");
    if (voxel != 0.0) {
        if (!h->params_set) return fail(MECH_E_STATE, "mech_set_params must come first");
        if (voxel < 2.0 * h->A * h->maxR * (1.0 + 1e-6))
            return fail(MECH_E_VOXEL_TOO_SMALL, "internal voxel must be >= 2 A max R (1 + 1e-6)");
    }
    h->voxel_int = voxel;
    h->grid_dirty = true;
    if (h->params_set) return build_grids(h);
    return MECH_OK;
}

int mech_set_launch(mech_t* h, int32_t force_block) {
    MECH_TRY(check_handle(h));
    if (force_block == 0) force_block = 256;
    if (force_block < 32 || force_block > 256 || force_block % 32)
        return fail(MECH_E_ARG, "force_block must be a multiple of 32 in [32, 256]");
    h->force_block = force_block;
    h->force_grid = h->sms * force_max_blocks_per_sm(h->mode, h->force_block);
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_set_tiling(mech_t* h, int32_t tile_x, int32_t tile_y, int32_t tile_z, int32_t dense_min) {
    MECH_TRY(check_handle(h));
    if (tile_x == 0 && tile_y == 0 && tile_z == 0) {
        h->use_tiles = false;
    } else {
        auto lg = [](int32_t v) { return v == 4 ? 2 : (v == 8 ? 3 : -1); };
        const int lx = lg(tile_x), ly = lg(tile_y), lz = lg(tile_z);
        if (!tile_shape_supported(lx, ly, lz))
            return fail(MECH_E_ARG, "supported tiles: 4x4x4, 4x4x8 or 8x4x4 voxels (or 0,0,0 to disable)");
        if (dense_min < 1) return fail(MECH_E_ARG, "dense_min must be >= 1");
        h->use_tiles = true;
        if (lx != h->ltx || ly != h->lty || lz != h->ltz) {
            h->ltx = lx;
            h->lty = ly;
            h->ltz = lz;
            h->grid_dirty = true;
        }
        h->dense_min = (uint32_t)dense_min;
    }
    h->invalidate_graphs();
    if (h->params_set && h->grid_dirty) return build_grids(h);
    return MECH_OK;
}

int mech_set_dense_kernel(mech_t* h, int32_t kernel) {
    MECH_TRY(check_handle(h));
    if (kernel != MECH_DENSE_WARP_PER_VOXEL && kernel != MECH_DENSE_BLOCK_PER_TILE)
        return fail(MECH_E_ARG, "dense kernel must be MECH_DENSE_WARP_PER_VOXEL or MECH_DENSE_BLOCK_PER_TILE");
    const int k = kernel == MECH_DENSE_WARP_PER_VOXEL ? kTileKernelVox : kTileKernelCTA;
    if (k != h->tile_kernel) {
        h->tile_kernel = k;
        h->tile_grid = tile_kernel_grid(h->args(0, 1), h->sms);
        h->invalidate_graphs();
    }
    return MECH_OK;
}

int mech_set_affinity(mech_t* h, int32_t ntypes, const double* aff) {
    MECH_TRY(check_handle(h));
    if (ntypes == 0 || !aff) {
        h->ntypes = 0;
        h->invalidate_graphs();
        return MECH_OK;
    }
    if (ntypes < 1 || ntypes > kMaxTypes) return fail(MECH_E_ARG, "ntypes must lie in [1, 16]");
    if (h->max_type >= ntypes)
        return fail(MECH_E_ARG, "a cell's type (" + std::to_string(h->max_type) + ") is outside the table");
    float tf[kMaxTypes * kMaxTypes];
    double td[kMaxTypes * kMaxTypes];
    for (int i = 0; i < kMaxTypes * kMaxTypes; ++i) {
        tf[i] = 1.0f;
        td[i] = 1.0;
    }
    for (int i = 0; i < ntypes; ++i)
        for (int j = 0; j < ntypes; ++j) {
            const double v = aff[i * ntypes + j];
            if (!std::isfinite(v)) return fail(MECH_E_NONFINITE, "non-finite affinity");
            if (v < 0.0) return fail(MECH_E_ARG, "affinities must be >= 0");
            if (v != aff[j * ntypes + i]) return fail(MECH_E_ARG, "the affinity matrix must be symmetric");
            td[i * kMaxTypes + j] = v;
            tf[i * kMaxTypes + j] = (float)v;
        }
    if (!h->d_aff_f) {
        MECH_TRY(h->alloc(&h->d_aff_f, (size_t)kMaxTypes * kMaxTypes));
        MECH_TRY(h->alloc(&h->d_aff_d, (size_t)kMaxTypes * kMaxTypes));
    }
    CUDA_TRY(cudaMemcpyAsync(h->d_aff_f, tf, sizeof(tf), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaMemcpyAsync(h->d_aff_d, td, sizeof(td), cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));  // the host tables die here
    h->ntypes = ntypes;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_set_walls(mech_t* h, int32_t face_mask, double c_wall) {
    MECH_TRY(check_handle(h));
    if (face_mask < 0 || face_mask > 63) return fail(MECH_E_ARG, "face_mask must lie in [0, 63]");
    if (!std::isfinite(c_wall)) return fail(MECH_E_NONFINITE, "non-finite wall coefficient");
    if (c_wall < 0.0) return fail(MECH_E_ARG, "the wall coefficient must be >= 0");
    h->walls = face_mask;
    h->c_wall = c_wall;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_set_stream(mech_t* h, void* stream) {
    MECH_TRY(check_handle(h));
    cudaStreamSynchronize(h->stream);
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return MECH_OK;
}

int mech_set_graph(mech_t* h, int32_t steps_per_graph) {
    MECH_TRY(check_handle(h));
    if (steps_per_graph < 0 || steps_per_graph % 2 || steps_per_graph > 100000)
        return fail(MECH_E_ARG, "steps_per_graph must be 0 or an even number <= 100000");
    h->graph_steps = steps_per_graph;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_set_precision(mech_t* h, int mode) {
    MECH_TRY(check_handle(h));
    if (mode != MECH_FP64 && mode != MECH_MIXED_FP64POS && mode != MECH_MIXED_KAHAN)
        return fail(MECH_E_ARG, "unknown precision mode");
    if (mode == h->mode) return MECH_OK;
    // value of positions and previous velocities -> io, switch, reload
    MECH_TRY(stage_out(h));
    h->mode = mode;
    StepArgs a = h->args(h->cur, 1);
    CUDA_TRY(launch_load_pos(a, h->st[h->cur], h->d_io, 0, nullptr, h->stream));
    CUDA_TRY(launch_load_vprev(a, h->st[h->cur], h->d_io + 3 * (size_t)h->npad, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->force_grid = h->sms * force_max_blocks_per_sm(h->mode, h->force_block);
    h->keys_valid = false;
    h->vout_valid = false;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_step(mech_t* h, int64_t n_steps) {
    MECH_TRY(ready(h));
    if (h->poisoned)
        return fail(MECH_E_STATE, "a device error left the state inconsistent; reload it with mech_load_state");
    if (n_steps < 0) return fail(MECH_E_ARG, "negative step count");
    if (n_steps == 0 || h->n == 0) {
        h->step += n_steps;
        return MECH_OK;
    }
    MECH_TRY(ensure_keys(h));
    h->vout_valid = false;
    while (!h->profiling && h->graph_steps > 0 && n_steps >= h->graph_steps) {
        if (!h->gexec[h->cur]) MECH_TRY(capture_graph(h));
        CUDA_TRY(cudaGraphLaunch(h->gexec[h->cur], h->stream));
        n_steps -= h->graph_steps;
        h->step += h->graph_steps;
    }
    for (int64_t s = 0; s < n_steps; ++s) {
        MECH_TRY(enqueue_step(h, 1, h->profiling));
        ++h->step;
    }
    return MECH_OK;
}

int mech_set_profiling(mech_t* h, int32_t enable) {
    MECH_TRY(check_handle(h));
    if (enable && h->prof_ev.empty()) {
        h->prof_ev.resize((size_t)mech::kProfCap * (mech::kProfPhases + 1), nullptr);
        for (cudaEvent_t& e : h->prof_ev) CUDA_TRY(cudaEventCreate(&e));
    }
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    h->profiling = enable != 0;
    h->prof_steps = 0;
    return MECH_OK;
}

int mech_read_profile(mech_t* h, double* phase_ms, int64_t* steps) {
    MECH_TRY(check_handle(h));
    if (!phase_ms) return fail(MECH_E_ARG, "null output");
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    for (int p = 0; p < mech::kProfPhases; ++p) phase_ms[p] = 0.0;
    for (int s = 0; s < h->prof_steps; ++s) {
        cudaEvent_t* ev = &h->prof_ev[(size_t)s * (mech::kProfPhases + 1)];
        for (int p = 0; p < mech::kProfPhases; ++p) {
            float ms = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&ms, ev[p], ev[p + 1]));
            phase_ms[p] += ms;
        }
    }
    if (steps) *steps = h->prof_steps;
    h->prof_steps = 0;
    return MECH_OK;
}

int mech_sync(mech_t* h) {
    MECH_TRY(check_handle(h));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return check_err_flag(h);
}

int mech_compute_velocities(mech_t* h, double* out3n) {
    MECH_TRY(ready(h));
    if (!out3n && h->n > 0) return fail(MECH_E_ARG, "null output");
    if (h->n == 0) return MECH_OK;
    MECH_TRY(ensure_keys(h));
    MECH_TRY(enqueue_step(h, 0));
    h->vout_valid = true;
    StepArgs a = h->args(h->cur, 0);
    const StateBuf& s = h->st[h->cur];
    if (h->mode == kFP64)
        CUDA_TRY(launch_unpermute_vel(a, s, nullptr, h->d_vout_d, h->d_io, h->stream));
    else
        CUDA_TRY(launch_unpermute_vel(a, s, h->d_vout_f, nullptr, h->d_io, h->stream));
    CUDA_TRY(cudaMemcpyAsync(out3n, h->d_io, 3 * (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream));
    return mech_sync(h);
}

int mech_read_positions(mech_t* h, double* out3n) {
    MECH_TRY(check_handle(h));
    if (h->n == 0) return MECH_OK;
    if (!out3n) return fail(MECH_E_ARG, "null output");
    StepArgs a = h->args(h->cur, 1);
    CUDA_TRY(launch_unpermute_pos(a, h->st[h->cur], h->d_io, h->d_io + 3 * (size_t)h->npad, h->d_tmp,
                                 8 * (size_t)h->npad, h->stream));
    CUDA_TRY(cudaMemcpyAsync(out3n, h->d_io, 3 * (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream));
    return mech_sync(h);
}

int mech_read_velocities(mech_t* h, double* out3n) {
    MECH_TRY(check_handle(h));
    if (h->n == 0) return MECH_OK;
    if (!out3n) return fail(MECH_E_ARG, "null output");
    StepArgs a = h->args(h->cur, 1);
    const StateBuf& s = h->st[h->cur];
    if (h->vout_valid) {
        if (h->mode == kFP64) CUDA_TRY(launch_unpermute_vel(a, s, nullptr, h->d_vout_d, h->d_io, h->stream));
        else CUDA_TRY(launch_unpermute_vel(a, s, h->d_vout_f, nullptr, h->d_io, h->stream));
    } else {
        if (h->mode == kFP64) CUDA_TRY(launch_unpermute_vel(a, s, nullptr, s.vp64, h->d_io, h->stream));
        else CUDA_TRY(launch_unpermute_vel(a, s, s.vpf, nullptr, h->d_io, h->stream));
    }
    CUDA_TRY(cudaMemcpyAsync(out3n, h->d_io, 3 * (size_t)h->n * 8, cudaMemcpyDeviceToHost, h->stream));
    return mech_sync(h);
}

int mech_write_positions(mech_t* h, const double* xyz3n) {
    MECH_TRY(check_handle(h));
    if (h->n == 0) return MECH_OK;
    if (!xyz3n) return fail(MECH_E_ARG, "null input");
    if (h->poisoned)
        return fail(MECH_E_STATE, "a device error left the state inconsistent; reload it with mech_load_state");
    CUDA_TRY(cudaMemcpyAsync(h->d_io, xyz3n, 3 * (size_t)h->n * 8, cudaMemcpyHostToDevice, h->stream));
    StepArgs a = h->args(h->cur, 1);
    CUDA_TRY(launch_load_pos(a, h->st[h->cur], h->d_io, 0, nullptr, h->stream));
    h->keys_valid = false;
    h->vout_valid = false;
    return MECH_OK;
}

int mech_read_state(mech_t* h, double* xyz, double* vprev, double* comp, int64_t* step) {
    MECH_TRY(check_handle(h));
    if (step) *step = h->step;
    if (h->n == 0) return MECH_OK;
    if (!xyz || !vprev) return fail(MECH_E_ARG, "null output");
    StepArgs a = h->args(h->cur, 1);
    const StateBuf& s = h->st[h->cur];
    const size_t n3 = 3 * (size_t)h->n * 8;
    double* io2 = h->d_io + 3 * (size_t)h->npad;
    if (h->mode == kMixedKahan) CUDA_TRY(launch_unpermute_vel(a, s, s.posf, nullptr, h->d_io, h->stream));
    else CUDA_TRY(launch_unpermute_vel(a, s, nullptr, s.pos64, h->d_io, h->stream));
    CUDA_TRY(cudaMemcpyAsync(xyz, h->d_io, n3, cudaMemcpyDeviceToHost, h->stream));
    if (h->mode == kFP64) CUDA_TRY(launch_unpermute_vel(a, s, nullptr, s.vp64, io2, h->stream));
    else CUDA_TRY(launch_unpermute_vel(a, s, s.vpf, nullptr, io2, h->stream));
    CUDA_TRY(cudaMemcpyAsync(vprev, io2, n3, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (comp) {
        if (h->mode == kMixedKahan) {
            CUDA_TRY(launch_unpermute_vel(a, s, s.comp, nullptr, h->d_io, h->stream));
            CUDA_TRY(cudaMemcpyAsync(comp, h->d_io, n3, cudaMemcpyDeviceToHost, h->stream));
        } else {
            std::memset(comp, 0, n3);
        }
    }
    return mech_sync(h);
}

int mech_load_state(mech_t* h, const double* xyz, const double* vprev, const double* comp, int64_t step) {
    MECH_TRY(check_handle(h));
    if (h->n > 0) {
        if (!xyz || !vprev) return fail(MECH_E_ARG, "null input");
        if (!finite_all(xyz, 3 * (size_t)h->n) || !finite_all(vprev, 3 * (size_t)h->n) ||
            (comp && !finite_all(comp, 3 * (size_t)h->n)))
            return fail(MECH_E_NONFINITE, "non-finite state");
        const size_t n3 = 3 * (size_t)h->n * 8;
        double* io2 = h->d_io + 3 * (size_t)h->npad;
        StepArgs a = h->args(h->cur, 1);
        CUDA_TRY(cudaMemcpyAsync(h->d_io, xyz, n3, cudaMemcpyHostToDevice, h->stream));
        if (comp && h->mode == kMixedKahan)
            CUDA_TRY(cudaMemcpyAsync(io2, comp, n3, cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(launch_load_pos(a, h->st[h->cur], h->d_io, 1, (comp && h->mode == kMixedKahan) ? io2 : nullptr,
                                 h->stream));
        CUDA_TRY(cudaMemcpyAsync(io2, vprev, n3, cudaMemcpyHostToDevice, h->stream));
        CUDA_TRY(launch_load_vprev(a, h->st[h->cur], io2, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
    }
    h->step = step;
    h->keys_valid = false;
    h->vout_valid = false;
    h->poisoned = false;
    return MECH_OK;
}

int mech_remove_cells(mech_t* h, const uint8_t* alive) {
    MECH_TRY(check_handle(h));
    if (h->poisoned)
        return fail(MECH_E_STATE, "a device error left the state inconsistent; reload it with mech_load_state");
    const uint32_t n = (uint32_t)h->n;
    if (n == 0) return MECH_OK;
    if (!alive) return fail(MECH_E_ARG, "null alive mask");
    // survivors per replicate (caller ranges): of a batch from the host mask;
    // of a single population from the device prefix sum below
    std::vector<int64_t> counts2(h->nrep, 0);
    int64_t n2 = 0;
    if (h->nrep > 1) {
        for (int r = 0; r < h->nrep; ++r)
            for (int64_t i = h->cbase[r]; i < h->cbase[r] + h->counts[r]; ++i) counts2[r] += alive[i] != 0;
        for (int64_t c : counts2) n2 += c;
        if (n2 == (int64_t)n) return MECH_OK;
    }
    // scratch for the two prefix sums (padded to the scan's tile)
    const size_t need = ((size_t)h->npad + kScanTile - 1) / kScanTile * kScanTile;
    if (h->ccap < need) {
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        h->free_ptr(h->d_alive, h->ccap);
        h->free_ptr(h->d_cflags, h->ccap * 4);
        h->free_ptr(h->d_cpref[0], h->ccap * 4);
        h->free_ptr(h->d_cpref[1], h->ccap * 4);
        h->free_ptr(h->d_cbsum, (h->ccap / kScanTile + 1) * 4);
        h->d_alive = nullptr;
        h->d_cflags = h->d_cpref[0] = h->d_cpref[1] = h->d_cbsum = nullptr;
        h->ccap = 0;
        int rc = h->alloc(&h->d_alive, need);
        if (rc == MECH_OK) rc = h->alloc(&h->d_cflags, need);
        if (rc == MECH_OK) rc = h->alloc(&h->d_cpref[0], need);
        if (rc == MECH_OK) rc = h->alloc(&h->d_cpref[1], need);
        if (rc == MECH_OK) rc = h->alloc(&h->d_cbsum, need / kScanTile + 1);
        if (rc != MECH_OK) return rc;
        h->ccap = need;
    }
    const uint32_t pad = (uint32_t)(((size_t)n + kScanTile - 1) / kScanTile * kScanTile);
    StepArgs a = h->args(h->cur, 1);
    uint32_t* newid = h->d_cpref[0];
    uint32_t* keep_pref = h->d_cpref[1];
    // new caller index of each survivor: exclusive prefix of the alive flags
    CUDA_TRY(cudaMemcpyAsync(h->d_alive, alive, n, cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(launch_alive_flags(h->d_alive, n, pad, h->d_cflags, h->stream));
    CUDA_TRY(launch_scan(h->d_cflags, pad, h->d_cbsum, newid, nullptr, nullptr, h->stream));
    if (h->nrep == 1) {
        uint32_t last[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(&last[0], newid + (n - 1), 4, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaMemcpyAsync(&last[1], h->d_cflags + (n - 1), 4, cudaMemcpyDeviceToHost, h->stream));
        CUDA_TRY(cudaStreamSynchronize(h->stream));
        n2 = (int64_t)last[0] + last[1];
        counts2[0] = n2;
        if (n2 == (int64_t)n) return MECH_OK;
    }
    // exclusive prefix of the keep flags in state order
    CUDA_TRY(launch_keep_flags(a, h->st[h->cur], h->d_alive, pad, h->d_cflags, h->stream));
    CUDA_TRY(launch_scan(h->d_cflags, pad, h->d_cbsum, keep_pref, nullptr, nullptr, h->stream));
    if (h->nrep == 1) {
        // one population: the survivors at or above n2 fill the dead slots below
        // it, in place (only as many cells move as died below n2)
        CUDA_TRY(launch_remove_in_place(a, h->d_alive, keep_pref, newid, (uint32_t)n2, h->d_cflags, h->stream));
    } else {
        // a batch: order-preserving compaction into the other state buffer, so
        // that every replicate stays one contiguous range
        CUDA_TRY(launch_compact_state(a, h->d_alive, keep_pref, newid, h->stream));
        h->cur ^= 1;
    }
    CUDA_TRY(launch_compact_params(a, h->d_alive, newid, h->d_io, h->stream));
    const size_t np = h->npad;
    if (n2 > 0) {
        CUDA_TRY(cudaMemcpyAsync(h->d_R64, h->d_io, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        CUDA_TRY(cudaMemcpyAsync(h->d_ccr64, h->d_io + np, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
        CUDA_TRY(cudaMemcpyAsync(h->d_cca64, h->d_io + 2 * np, n2 * 8, cudaMemcpyDeviceToDevice, h->stream));
    }
    MECH_TRY(set_cell_counts(h, counts2));
    return mech_sync(h);
}

// New cells: per_rep[r] of them for replicate r (all of them for a single
// population), given in replicate order.
static int add_cells(mech_t* h, const int64_t* per_rep, int64_t m, const double* xyz, const double* R,
                     const double* ccr, const double* cca, const int32_t* type) {
    MECH_TRY(check_handle(h));
    if (h->poisoned)
        return fail(MECH_E_STATE, "a device error left the state inconsistent; reload it with mech_load_state");
    if (m < 0) return fail(MECH_E_ARG, "negative cell count");
    std::vector<int64_t> add(h->nrep, 0);
    if (per_rep) {
        int64_t s = 0;
        for (int r = 0; r < h->nrep; ++r) {
            if (per_rep[r] < 0) return fail(MECH_E_ARG, "negative cell count for a replicate");
            add[r] = per_rep[r];
            s += per_rep[r];
        }
        if (s != m) return fail(MECH_E_ARG, "per-replicate counts do not add up to m");
    } else {
        add[0] = m;
    }
    if (m == 0) return MECH_OK;
    MECH_TRY(validate_cells(m, xyz, R, ccr, cca));
    int32_t max_type = -1;
    MECH_TRY(check_types(m, type, max_type));
    if (h->ntypes > 0 && max_type >= h->ntypes)
        return fail(MECH_E_ARG, "a new cell's type is outside the affinity table (mech_set_affinity)");
    if (h->n + m >= (int64_t)0x7FFFFFFF) return fail(MECH_E_ARG, "more than 2^31-1 cells");
    double maxR = h->maxR;
    for (int64_t i = 0; i < m; ++i) maxR = std::max(maxR, R[i]);
    if (h->params_set && maxR > h->maxR) {
        if (h->voxel_user < 2.0 * h->A * maxR)
            return fail(MECH_E_VOXEL_TOO_SMALL, "a new radius needs voxel_size >= 2 A max R = " +
                                                    std::to_string(2.0 * h->A * maxR));
        if (h->voxel_int > 0.0 && h->voxel_int < 2.0 * h->A * maxR * (1.0 + 1e-6))
            return fail(MECH_E_VOXEL_TOO_SMALL, "a new radius needs an internal voxel >= 2 A max R (1 + 1e-6)");
    }
    const int64_t n = h->n;
    if ((size_t)(n + m) > (size_t)h->npad) {
        const size_t cap2 = (size_t)(std::max<int64_t>(n + m, n + n / 2) + 63) / 64 * 64;
        MECH_TRY(grow_capacity(h, cap2));
    }
    cudaStream_t st = h->stream;
    const size_t np = h->npad;
    // replicate r's cells move up by the cells added before it
    std::vector<uint32_t> shift(h->nrep, 0);
    bool shifted = false;
    for (int r = 1; r < h->nrep; ++r) {
        shift[r] = shift[r - 1] + (uint32_t)add[r - 1];
        shifted = shifted || (shift[r] > 0 && h->counts[r] > 0);
    }
    if (shifted) {
        if (h->shift_cap < (size_t)h->nrep) {
            h->free_ptr(h->d_shift, h->shift_cap * 4);
            h->d_shift = nullptr;
            h->shift_cap = 0;
            MECH_TRY(h->alloc(&h->d_shift, (size_t)h->nrep));
            h->shift_cap = (size_t)h->nrep;
        }
        CUDA_TRY(cudaMemcpyAsync(h->d_shift, shift.data(), h->nrep * 4, cudaMemcpyHostToDevice, st));
        StepArgs a = h->args(h->cur, 1);
        CUDA_TRY(launch_shift(a, h->d_shift, h->d_io, st));
        h->cur ^= 1;
        CUDA_TRY(cudaMemcpyAsync(h->d_R64, h->d_io, (n + m) * 8, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(h->d_ccr64, h->d_io + np, (n + m) * 8, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaMemcpyAsync(h->d_cca64, h->d_io + 2 * np, (n + m) * 8, cudaMemcpyDeviceToDevice, st));
    }
    // slot (= caller index) of every new cell: after its replicate's cells
    std::vector<uint32_t> dst(m);
    std::vector<int64_t> counts2(h->nrep);
    int64_t k = 0, base = 0;
    for (int r = 0; r < h->nrep; ++r) {
        for (int64_t j = 0; j < add[r]; ++j) dst[k++] = (uint32_t)(base + h->counts[r] + j);
        counts2[r] = h->counts[r] + add[r];
        base += counts2[r];
    }
    // new cells' positions and parameters, packed in io; dst in perm (binning
    // scratch, free between steps)
    CUDA_TRY(cudaMemcpyAsync(h->d_io, xyz, 3 * m * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_io + 3 * m, R, m * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_io + 4 * m, ccr, m * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_io + 5 * m, cca, m * 8, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(h->d_perm, dst.data(), m * 4, cudaMemcpyHostToDevice, st));
    // types in the key scratch (the next step recomputes the keys)
    if (type) CUDA_TRY(cudaMemcpyAsync(h->d_key, type, m * 4, cudaMemcpyHostToDevice, st));
    CUDA_TRY(launch_append_state(h->args(h->cur, 1), h->st[h->cur], h->d_io, h->d_perm,
                                 type ? reinterpret_cast<const uint32_t*>(h->d_key) : nullptr,
                                 (uint32_t)m, h->d_R64, h->d_ccr64, h->d_cca64, st));
    CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors above and the caller's arrays are released
    h->maxR = maxR;
    h->max_type = std::max(h->max_type, max_type);
    h->keys_valid = false;
    MECH_TRY(set_cell_counts(h, counts2));
    return mech_sync(h);
}

int mech_add_cells(mech_t* h, int64_t m, const double* xyz, const double* R, const double* ccr, const double* cca,
                   const int32_t* type) {
    MECH_TRY(check_handle(h));
    if (h->nrep != 1) return fail(MECH_E_ARG, "mech_add_cells: use mech_add_cells_batch for a batch handle");
    return add_cells(h, nullptr, m, xyz, R, ccr, cca, type);
}

int mech_add_cells_batch(mech_t* h, const int64_t* counts, const double* xyz, const double* R, const double* ccr,
                         const double* cca, const int32_t* type) {
    MECH_TRY(check_handle(h));
    if (!counts) return fail(MECH_E_ARG, "null counts");
    int64_t m = 0;
    for (int r = 0; r < h->nrep; ++r) m += counts[r];
    return add_cells(h, counts, m, xyz, R, ccr, cca, type);
}

int mech_debug_bins(mech_t* h, uint32_t* key, uint32_t* count, uint32_t* start, int64_t* order) {
    MECH_TRY(ready(h));
    if (h->n == 0) {
        if (count) std::memset(count, 0, (size_t)h->V * 4);
        if (start) std::memset(start, 0, ((size_t)h->V + 1) * 4);
        return MECH_OK;
    }
    h->keys_valid = false;
    MECH_TRY(ensure_keys(h));
    StepArgs a = h->args(h->cur, 1);
    CUDA_TRY(launch_scan(a.count_cur, h->Vpad, h->d_bsum, h->d_start, nullptr, h->d_occ, h->stream));
    // the scatter counts the histogram back down to zero: copy it first
    if (count) CUDA_TRY(cudaMemcpyAsync(count, a.count_cur, (size_t)h->V * 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(launch_scatter(a, h->elem_grid, h->stream));
    CUDA_TRY(launch_canon(a, h->elem_grid, h->stream));
    h->keys_valid = false;
    const size_t n = (size_t)h->n;
    std::vector<uint32_t> k(n), ids(n), perm(n);
    CUDA_TRY(cudaMemcpyAsync(k.data(), h->d_key, n * 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(ids.data(), h->st[h->cur].id, n * 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaMemcpyAsync(perm.data(), h->d_perm, n * 4, cudaMemcpyDeviceToHost, h->stream));
    if (start) CUDA_TRY(cudaMemcpyAsync(start, h->d_start, ((size_t)h->V + 1) * 4, cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    if (key)
        for (size_t i = 0; i < n; ++i) key[ids[i]] = k[i];
    if (order)
        for (size_t f = 0; f < n; ++f) order[f] = ids[perm[f]];
    return check_err_flag(h);
}

int mech_pair_stats(mech_t* h, int64_t* candidates, int64_t* pairs) {
    MECH_TRY(ready(h));
    if (candidates) *candidates = 0;
    if (pairs) *pairs = 0;
    if (h->n == 0) return MECH_OK;
    if (h->poisoned)
        return fail(MECH_E_STATE, "a device error left the state inconsistent; reload it with mech_load_state");
    // FP64 positions in caller order, then a binning pass into the B buffers
    StepArgs a = h->args(h->cur, 1);
    CUDA_TRY(launch_unpermute_pos(a, h->st[h->cur], h->d_io, h->d_io + 3 * (size_t)h->npad, h->d_tmp,
                                 8 * (size_t)h->npad, h->stream));
    h->keys_valid = false;
    MECH_TRY(ensure_keys(h));
    CUDA_TRY(launch_scan(a.count_cur, h->Vpad, h->d_bsum, h->d_start, nullptr, h->d_occ, h->stream));
    CUDA_TRY(launch_scatter(a, h->elem_grid, h->stream));
    CUDA_TRY(launch_canon(a, h->elem_grid, h->stream));
    h->keys_valid = false;  // the scatter counted the histogram down
    CUDA_TRY(cudaMemsetAsync(h->d_stats, 0, 2 * sizeof(unsigned long long), h->stream));
    CUDA_TRY(launch_pair_stats(a, h->d_io, h->d_stats, h->sms * 8, h->stream));
    unsigned long long c[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(c, h->d_stats, sizeof(c), cudaMemcpyDeviceToHost, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    MECH_TRY(check_err_flag(h));
    if (candidates) *candidates = (int64_t)c[0];
    if (pairs) *pairs = (int64_t)(c[1] / 2);
    return MECH_OK;
}

int mech_debug_inject(mech_t* h, int32_t fault) {
    if (fault == MECH_FAULT_ALLOC) {
        g_fault_alloc.store(1);
        return MECH_OK;
    }
    if (fault == MECH_FAULT_NONE) {
        g_fault_alloc.store(0);
        if (!h) return MECH_OK;
    }
    MECH_TRY(check_handle(h));
    if (fault != MECH_FAULT_NONE && fault != MECH_FAULT_TILE_WAIT) return fail(MECH_E_ARG, "unknown fault");
    h->fault = fault == MECH_FAULT_TILE_WAIT ? kFaultTileWait : 0u;
    h->invalidate_graphs();
    return MECH_OK;
}

int mech_info(mech_t* h, mech_info_t* out) {
    MECH_TRY(check_handle(h));
    if (!out) return fail(MECH_E_ARG, "null output");
    if (h->params_set && h->grid_dirty) MECH_TRY(build_grids(h));
    std::memset(out, 0, sizeof(*out));
    out->n_cells = h->n;
    out->n_rep = h->nrep;
    out->mode = h->mode;
    out->n_voxels = h->V;
    if (!h->grids.empty())
        for (int d = 0; d < 3; ++d) out->dims[d] = h->grids[0].n[d];
    out->voxel = voxel_of(h);
    out->step = h->step;
    out->launches_per_step = h->n > 0 ? ((h->mode != kFP64 && h->use_tiles) ? 8 : 6) : 0;
    out->graph_steps = h->graph_steps;
    out->device_bytes = (int64_t)h->dev_bytes;
    return MECH_OK;
}

int mech_grid(mech_t* h, int32_t rep, double* lo3, int32_t* dims3, int64_t* voxel_base) {
    MECH_TRY(check_handle(h));
    if (rep < 0 || rep >= h->nrep) return fail(MECH_E_ARG, "replicate index out of range");
    if (!h->params_set) return fail(MECH_E_STATE, "mech_set_params must come first");
    if (h->grid_dirty) MECH_TRY(build_grids(h));
    const GridDev& g = h->grids[rep];
    for (int d = 0; d < 3; ++d) {
        if (lo3) lo3[d] = g.lo[d];
        if (dims3) dims3[d] = g.n[d];
    }
    if (voxel_base) *voxel_base = g.vbase;
    return MECH_OK;
}

int mech_destroy(mech_t* h) {
    if (!h) return MECH_OK;
    if (h->stream) cudaStreamSynchronize(h->stream);
    delete h;
    return MECH_OK;
}

}  // extern "C"
