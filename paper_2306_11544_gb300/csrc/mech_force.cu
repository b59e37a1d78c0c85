// Neighbour-gather velocity and AB2 integration (steps 2 and 3 of the
// mechanics update; the paper's "update velocity" region, Sec. 5.4).
//
// Mixed precision modes run four launches per step:
//   k_tile_classify   flags every voxel tile (TX x TY x TZ voxels) holding at
//                     least `dense_min` cells and lists the flagged tiles;
//   k_force_tile      one CTA per dense tile (CTAs claim tiles one at a time
//                     from a cursor): the rows of the tile's halo (one voxel
//                     around it) are contiguous runs of the voxel-sorted
//                     force records, so each row is staged into shared
//                     memory by one TMA bulk copy; then one thread per
//                     target cell tests its 27-voxel neighbourhood there;
//   k_sparse_list     lists the cells outside dense tiles;
//   k_force_cells     one thread per listed cell (sparse regions), reading
//                     its neighbours through L1.
// The split is the GPU form of the paper's load-balance lesson (Sec. 5.4):
// work follows voxel occupancy, dense regions are computed tile by tile in
// mesh order (the coarse, cache-friendly grain the paper recommends) and empty
// voxels cost nothing.
//
// Candidate tests compare the hi-part distance with A (R_i + R_j) plus a
// margin of 2q (about 12 FP32 instructions per candidate); in the tile kernel
// the tests of 32 candidates set bits of a hit mask and only the hits are then
// evaluated exactly, so the pair term never runs inside the scan.
// Every cell's sum is taken in the same candidate order: (dz, dy) rows in
// lexicographic order, cells in voxel order inside a row.
//
// Record positions are relative to the grid centre, split into a hi part on a
// power-of-two grid q (differences of hi parts are exact) and a residual; the
// pair vector (hi_i - hi_j) + (lo_i - lo_j) is exact up to its final rounding,
// and records are used as staged, with no per-tile frame shift.  No FP64
// arithmetic runs in any candidate loop (FP64 is ~1/62 of FP32 throughput on
// this GPU).
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "mech_internal.cuh"

namespace mk {

namespace {

constexpr int kCellBlock = 256;
constexpr uint32_t kSpinLimit = 1u << 26;

struct Cell3 {
    int ix, iy, iz;
};

__device__ __forceinline__ Cell3 decode(uint32_t k, const GridDev& g) {
    const uint32_t local = k - g.vbase;
    Cell3 c;
    c.ix = (int)(local % (uint32_t)g.n[0]);
    const uint32_t rest = local / (uint32_t)g.n[0];
    c.iy = (int)(rest % (uint32_t)g.n[1]);
    c.iz = (int)(rest / (uint32_t)g.n[1]);
    return c;
}

// ------------------------------------------------------- PTX helpers ----

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion counted on `bar`.
// Requires 16-byte aligned addresses and a size that is a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of the barrier; give up after `limit_ns` of wall
// time (or kSpinLimit tries, whichever comes first).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 0; i < kSpinLimit; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// ------------------------------------------------- shared arithmetic ----

// Velocity sum with a Kahan compensation term per component: the sum of a
// cell's pair terms is free of the cancellation error of a plain FP32 sum
// (pair terms of a cell near force balance are much larger than their sum).
struct Acc3 {
    float x, y, z, cx, cy, cz;
    __device__ __forceinline__ void zero() { x = y = z = cx = cy = cz = 0.f; }
    __device__ __forceinline__ static void add1(float& s, float& c, float v) {
        const float u = __fsub_rn(v, c);
        const float t = __fadd_rn(s, u);
        c = __fsub_rn(__fsub_rn(t, s), u);
        s = t;
    }
    __device__ __forceinline__ void add(float vx, float vy, float vz) {
        add1(x, cx, vx);
        add1(y, cy, vy);
        add1(z, cz, vz);
    }
    __device__ __forceinline__ float vx() const { return __fsub_rn(x, cx); }
    __device__ __forceinline__ float vy() const { return __fsub_rn(y, cy); }
    __device__ __forceinline__ float vz() const { return __fsub_rn(z, cz); }
};

// Approximate FP32 reciprocal square root and quotient in their PTX forms
// that flush subnormal operands and results to zero (no scaling path for
// them): d^2 > 0 is checked first and S (S + d) is of the order of R^2, so
// no operand of the pair term is subnormal, and a subnormal quotient would
// stand for a term below 1e-38.  For normal values the results equal those
// of rsqrtf and __fdividef.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float div_ftz(float a, float b) {
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// Pair term (FP32) for a candidate at offset r = x_i - x_j, given as an exact
// hi part h (a difference of values on the q grid) plus a small lo part l;
// Rlo is the sum of the two radius residuals R - (float)R.  Sets f to
// (c_r - c_a) r / d and returns true if 0 < d < A S (else f = 0, false).
//   1 - d/S is formed as (S^2 - d^2) / (S (S + d)), with d^2 and S^2 carried
//   as unevaluated sums (error-free products and sums), so the cancellation of
//   1 - d/S near contact costs no accuracy: t and t_a are accurate to a few
//   ulp even where d/S is close to 1, which a direct 1 - d/S is not.  The
//   adhesion term uses (A S)^2 - d^2 = S^2 (A^2 - 1) + (S^2 - d^2), A2m1 being
//   A^2 - 1 rounded once.
__device__ __forceinline__ bool pair_force(float hx, float hy, float hz, float lx, float ly, float lz, float Ri,
                                           float Rj, float Rlo, float sccri, float sccai, float sccrj, float sccaj,
                                           float aij, float A, float A2m1, float3& f) {
    const float rx = hx + lx, ry = hy + ly, rz = hz + lz;
    const float d2 = rx * rx + ry * ry + rz * rz;
    float Se;
    const float S = two_sum(Ri, Rj, Se);  // S + Se == Ri + Rj
    Se += Rlo;
    const float AS = A * S;
    if (d2 < AS * AS && d2 > 0.f) {
        // d^2 = D + De
        const float px = hx * hx, py = hy * hy, pz = hz * hz;
        float e1, e2;
        const float D1 = two_sum(px, py, e1);
        const float D = two_sum(D1, pz, e2);
        const float De = ((fmaf(hx, hx, -px) + fmaf(hy, hy, -py)) + (fmaf(hz, hz, -pz) + (e1 + e2))) +
                         (lx * (2.f * hx + lx) + ly * (2.f * hy + ly) + lz * (2.f * hz + lz));
        const float rd = rsqrt_ftz(d2);
        const float d = d2 * rd;
        // g = S^2 - d^2, with S^2 = S2 + eS; then (A S)^2 - d^2 = S^2 (A^2 - 1) + g
        const float S2 = S * S;
        const float eS = fmaf(S, S, -S2) + 2.f * S * Se;
        const float g = (S2 - D) + (eS - De);
        const float gA = fmaf(S2, A2m1, fmaf(eS, A2m1, g));
        const float ta = div_ftz(gA, AS * (AS + d));
        float cf = -(aij * (sccai * sccaj)) * (ta * ta);
        // repulsion for d < S, as a select: the lanes of a warp's hit loop
        // then run one path (S (S + d) > 0, so the unused quotient is finite)
        const float t = div_ftz(g, S * (S + d));
        const float cr = cf + (sccri * sccrj) * (t * t);
        cf = d < S ? cr : cf;
        const float sc = cf * rd;
        f = make_float3(sc * rx, sc * ry, sc * rz);
        return true;
    }
    f = make_float3(0.f, 0.f, 0.f);
    return false;
}

__device__ __forceinline__ void pair_term(float hx, float hy, float hz, float lx, float ly, float lz, float Ri,
                                          float Rj, float Rlo, float sccri, float sccai, float sccrj, float sccaj,
                                          float aij, float A, float A2m1, Acc3& acc) {
    float3 f;
    if (pair_force(hx, hy, hz, lx, ly, lz, Ri, Rj, Rlo, sccri, sccai, sccrj, sccaj, aij, A, A2m1, f))
        acc.add(f.x, f.y, f.z);
}

// Squared candidate cutoff for a target with cut_i = A R_i + margin.
__device__ __forceinline__ bool candidate_hit(float hx, float hy, float hz, float A, float Rj, float cut_i) {
    const float c = fmaf(A, Rj, cut_i);
    return hx * hx + hy * hy + hz * hz < c * c;
}

// State that the AB2 update of a cell reads: previous velocity and position
// (FP64, or FP32 x_hi with its compensation), from the A order.
template <int MODE>
struct CellState {
    float vp[3];
    float xh[3], cc[3];  // Kahan mode
    double x[3];         // FP64-position mode
};

// Position in the A (previous) order of the cell at B position q.
__device__ __forceinline__ uint32_t a_slot(const StepArgs& a, uint32_t q) {
    uint32_t src = a.perm[q];
    if (src >= a.n) {  // only after an earlier device error
        atomicOr(a.err, kErrIndex);
        src = q;
    }
    return src;
}

// The state is read where the previous step left it (A order, slot src =
// perm[q]): the canonicalisation moves only the force records into B order.
template <int MODE>
__device__ __forceinline__ CellState<MODE> load_cell_state(const StepArgs& a, uint32_t src) {
    const size_t np = a.npad;
    CellState<MODE> st;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.vp[d] = a.A.vpf[d * np + src];
        if (MODE == kMixedFP64Pos) {
            st.x[d] = a.A.pos64[d * np + src];
        } else {
            st.xh[d] = a.A.posf[d * np + src];
            st.cc[d] = a.A.comp[d * np + src];
        }
    }
    return st;
}

// AB2 update of cell q: state st read from the A order, new state written at q
// in the B order; returns the next step's voxel key and its voxel coordinates.
template <int MODE>
__device__ __forceinline__ uint32_t ab2_apply(const StepArgs& a, const GridDev& g, uint32_t q,
                                              const CellState<MODE>& st, float ax, float ay, float az, float Rf,
                                              float Rlo, int& nix, int& niy, int& niz) {
    const size_t np = a.npad;
    float v[3] = {ax, ay, az};
    if (a.walls) {  // wall terms (velocity variant): an FP32 test, then FP64 for cells near a face
        float x0[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) x0[d] = MODE == kMixedFP64Pos ? __double2float_rn(st.x[d]) : st.xh[d];
        if (near_wall(a, g, x0, Rf)) {
            double x[3], w[3] = {0.0, 0.0, 0.0};
#pragma unroll
            for (int d = 0; d < 3; ++d)
                x[d] = MODE == kMixedFP64Pos ? st.x[d] : __dsub_rn((double)st.xh[d], (double)st.cc[d]);
            wall_terms(a, g, x, __dadd_rn((double)Rf, (double)Rlo), w);
#pragma unroll
            for (int d = 0; d < 3; ++d) v[d] = __fadd_rn(v[d], __double2float_rn(w[d]));
        }
    }
    bool finite = true;
    float xf[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float inc = a.dt_f * (1.5f * v[d] - 0.5f * st.vp[d]);
        // the whole state is written in B order; a velocities-only pass
        // (integrate 0) writes it unchanged
        if (MODE == kMixedFP64Pos) {
            const double xn = a.integrate ? __dadd_rn(st.x[d], (double)inc) : st.x[d];
            a.B.pos64[d * np + q] = xn;
            xf[d] = __double2float_rn(xn);
            finite = finite && isfinite(xn);
        } else {
            float xh = st.xh[d], cc = st.cc[d];
            if (a.integrate) {
                const float y = __fsub_rn(inc, cc);
                const float t = __fadd_rn(xh, y);
                cc = __fsub_rn(__fsub_rn(t, xh), y);
                xh = t;
            }
            a.B.posf[d * np + q] = xh;
            a.B.comp[d * np + q] = cc;
            xf[d] = xh;
            finite = finite && isfinite(xh);
        }
        a.B.vpf[d * np + q] = a.integrate ? v[d] : st.vp[d];
        if (!a.integrate) a.vout_f[d * np + q] = v[d];
        finite = finite && isfinite(v[d]);
    }
    if (!finite) atomicOr(a.err, kErrNonFinite);
    nix = axis_index_f32(xf[0], g.lo_f[0], g.inv_h_f, g.n[0]);
    niy = axis_index_f32(xf[1], g.lo_f[1], g.inv_h_f, g.n[1]);
    niz = axis_index_f32(xf[2], g.lo_f[2], g.inv_h_f, g.n[2]);
    return g.vbase + (uint32_t)nix + (uint32_t)g.n[0] * ((uint32_t)niy + (uint32_t)g.n[1] * (uint32_t)niz);
}

template <int MODE>
__device__ __forceinline__ uint32_t ab2_epilogue(const StepArgs& a, const GridDev& g, uint32_t q, uint32_t src,
                                                 float ax, float ay, float az, float Rf, float Rlo, int& nix,
                                                 int& niy, int& niz) {
    const CellState<MODE> st = load_cell_state<MODE>(a, src);
    return ab2_apply<MODE>(a, g, q, st, ax, ay, az, Rf, Rlo, nix, niy, niz);
}

// Next-step histograms (voxels, scan blocks, tiles) and key of cell q; all 32
// lanes call it.
__device__ __forceinline__ void next_step_counts(const StepArgs& a, uint32_t q, uint32_t nkey, uint32_t ntile,
                                                 bool valid) {
    warp_add(a.tcount_nxt, ntile, valid);  // many lanes share a tile: aggregate
    warp_add(a.bcount_nxt, nkey / (uint32_t)kScanTile, valid);  // and a scan block
    if (valid) {
        atomicAdd(&a.count_nxt[nkey], 1u);  // voxels hold ~2 cells: plain reduction
        a.key[q] = nkey;
    }
}

// Velocity of cell q by a direct walk over its 27 neighbour voxels in global
// memory (L1-cached).  Candidate order: (dz, dy) rows, then voxel order.  The
// occupancy bits of all nine rows are fetched first (independent loads), so
// a cell with few or no neighbours costs one round of memory latency, not nine.
// A cell alone in its voxel leaves that voxel out (it holds only the skipped
// self pair), so an isolated cell walks no run at all.  Candidates are tested
// on the hi parts; a pair that passes is evaluated from hi + lo.
template <bool AFF>
__device__ __forceinline__ void velocity_walk(const StepArgs& a, const GridDev& g, const Cell3& c, uint32_t q,
                                              bool alone, const float4 pi, const float4 qi, Acc3& acc) {
    const float A = a.A_f;
    const int jx0 = c.ix > 0 ? c.ix - 1 : 0;
    const int jx1 = c.ix + 1 < g.n[0] ? c.ix + 1 : g.n[0] - 1;
    const uint32_t wmask = (1u << (jx1 - jx0 + 1)) - 1u;
    uint32_t occ9 = 0u;  // 3 occupancy bits per (dz, dy) row, row p at bits 3p..3p+2
#pragma unroll
    for (int p = 0; p < 9; ++p) {
        const int jz = c.iz + p / 3 - 1, jy = c.iy + p % 3 - 1;
        if (jz >= 0 && jz < g.n[2] && jy >= 0 && jy < g.n[1]) {
            const uint32_t row = g.vbase + (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
            const uint32_t b0 = row + (uint32_t)jx0, sh = b0 & 31u;
            uint32_t w = a.occ[b0 >> 5] >> sh;
            if (sh > 29u) w |= a.occ[(b0 >> 5) + 1] << (32u - sh);
            occ9 |= (w & wmask) << (3 * p);
        }
    }
    if (alone) occ9 &= ~(1u << (12 + (c.ix - jx0)));  // own voxel: row (dz, dy) = (0, 0) is row 4
    const float4 li = record_lo(pi, qi, g.qs);
    const float cut_i = fmaf(A, pi.w, g.qm + a.cut_eps);
    acc.zero();
    // One iteration per run of occupied voxels in a row, lowest bit first: rows
    // (dz, dy) in lexicographic order, voxels along x inside a row (the
    // candidate order).  A run's cells are one contiguous range of the sorted
    // records, so it needs two start[] entries.  A warp's sequential steps are
    // then its lanes' largest run count, not the union of their occupied voxels.
    uint32_t bits = occ9;
    while (bits) {
        const int b = __ffs(bits) - 1;
        const int p = b / 3, o = b - 3 * p;
        const uint32_t run = (bits >> b) & (7u >> o);   // this row's remaining bits from o
        const int len = __ffs(~run) - 1;                // consecutive occupied voxels (1..3)
        bits &= ~(((1u << len) - 1u) << b);
        const int jz = c.iz + p / 3 - 1, jy = c.iy + p % 3 - 1;
        const uint32_t v0 = g.vbase + (uint32_t)(jx0 + o) +
                            (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
        {
            const uint32_t s = a.start[v0], e = a.start[v0 + (uint32_t)len];
            for (uint32_t j = s; j < e; ++j) {
                const float4 pj = a.B.rec[2 * (size_t)j];
                const float hx = pi.x - pj.x, hy = pi.y - pj.y, hz = pi.z - pj.z;
                if (j != q && candidate_hit(hx, hy, hz, A, pj.w, cut_i)) {
                    const float4 qj = a.B.rec[2 * (size_t)j + 1];
                    const float4 lj = record_lo(pj, qj, g.qs);
                    const float aij = AFF ? __ldg(&a.aff_f[record_type(qi) * kMaxTypes + record_type(qj)]) : 1.0f;
                    pair_term(hx, hy, hz, li.x - lj.x, li.y - lj.y, li.z - lj.z, pi.w, pj.w, li.w + lj.w, qi.x, qi.y,
                              qj.x, qj.y, aij, A, a.A2m1_f, acc);
                }
            }
        }
    }
}

// ------------------------------------------- thread-per-cell kernel ----
// Every cell not owned by a dense tile: the cells listed by k_sparse_list, or
// all cells when tiles are off.  (Claiming 32 listed cells at a time from a
// cursor instead of the static grid-stride assignment measured slower: the
// claim's round trip lengthens every iteration of this latency-bound loop.)
template <int MODE, bool AFF>
__global__ void __launch_bounds__(kCellBlock, 4) k_force_cells(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t total = a.use_tiles ? a.nsparse[0] : a.n;
    // the list entry (or key) of the next iteration is loaded one iteration
    // ahead, so an iteration's chain of dependent loads starts one step later
    auto entry = [&](uint32_t idx) -> uint2 {
        if (idx >= total) return make_uint2(0u, 0u);
        return a.use_tiles ? a.slist[idx] : make_uint2(idx, a.vkey_s[idx]);
    };
    uint2 next = entry(warp * 32u + lane);
    for (uint32_t base = warp * 32u; base < total; base += nwarps * 32u) {
        const uint32_t idx = base + lane;
        const bool valid = idx < total;
        const uint2 e = next;
        next = entry(idx + nwarps * 32u);
        uint32_t q = 0, nkey = 0, ntile = 0;
        if (valid) {
            q = e.x & 0x7FFFFFFFu;
            const bool alone = (e.x >> 31) != 0u;  // only set in list entries
            const uint32_t key = e.y;
            const CellState<MODE> st = load_cell_state<MODE>(a, a_slot(a, q));  // issued before the walk
            const int r = rep_of_cell(a.grids, a.nrep, q);
            const GridDev& g = a.grids[r];
            const Cell3 c = decode(key, g);
            Acc3 acc;
            velocity_walk<AFF>(a, g, c, q, alone, a.B.rec[2 * (size_t)q], a.B.rec[2 * (size_t)q + 1], acc);
            float Rf = 0.f, Rlo = 0.f;  // the radius, for the wall terms only
            if (a.walls) {
                const float4 pq = a.B.rec[2 * (size_t)q], cq = a.B.rec[2 * (size_t)q + 1];
                Rf = pq.w;
                Rlo = record_lo(pq, cq, g.qs).w;
            }
            int nix, niy, niz;
            nkey = ab2_apply<MODE>(a, g, q, st, acc.vx(), acc.vy(), acc.vz(), Rf, Rlo, nix, niy, niz);
            ntile = tile_index(g, nix, niy, niz, a.ltx, a.lty, a.ltz);
        }
        next_step_counts(a, q, nkey, ntile, valid);
    }
}

// A tile is processed by the tile kernel only when its whole halo lies inside
// the grid (1 <= b and T b + T <= n - 1 on every axis, T the tile's extent):
// the kernel's shape is then fixed (6 x (TZ + 2) halo rows of TX + 2 voxels
// around TX x 4 x TZ core voxels) and its index arithmetic compiles to
// constants.
// Tiles at the grid faces go to the thread-per-cell kernel.
__device__ __forceinline__ bool tile_interior(const GridDev& g, int bx, int by, int bz, int tx, int tz) {
    return bx >= 1 && by >= 1 && bz >= 1 && tx * bx + tx <= g.n[0] - 1 && 4 * by + 4 <= g.n[1] - 1 &&
           tz * bz + tz <= g.n[2] - 1;
}

// ----------------------------------------------------- tile classify ----
// Flags dense tiles, lists them, clears the next step's tile histogram and the
// sparse-cell counter.
__global__ void k_tile_classify(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.nsparse[0] = 0u;  // sparse-list length
        a.nsparse[1] = 0u;  // tile cursor of the tile kernel
    }
    for (uint32_t base = warp * 32u; base < a.ntiles; base += nwarps * 32u) {
        const uint32_t t = base + lane;
        const bool valid = t < a.ntiles;
        bool dense = false;
        if (valid) {
            dense = a.use_tiles && a.tcount_cur[t] >= a.dense_min;
            if (dense && a.tile_kernel == kTileKernelCTA) {
                const int r = rep_of_tile(a.grids, a.nrep, t);
                const GridDev& g = a.grids[r];
                const uint32_t lt = t - g.tbase;
                const uint32_t rest = lt / (uint32_t)g.nt[0];
                dense = tile_interior(g, (int)(lt % (uint32_t)g.nt[0]), (int)(rest % (uint32_t)g.nt[1]),
                                      (int)(rest / (uint32_t)g.nt[1]), 1 << a.ltx, 1 << a.ltz);
            }
            a.tdense[t] = dense ? 1 : 0;
            a.tcount_nxt[t] = 0u;
        }
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, dense);
        uint32_t off = 0;
        if (lane == 0 && m) off = atomicAdd(a.ndense, (uint32_t)__popc(m));
        off = __shfl_sync(0xFFFFFFFFu, off, 0);
        if (dense) a.tlist[off + __popc(m & lanemask_lt())] = t;
    }
}

// ------------------------------------------------- voxel-warp kernel ----
// Dense tiles, one warp per tile at a time (warps claim tiles from a cursor;
// no block-level barrier anywhere, warps run independently), voxel by voxel
// in mesh order (x fastest).  For one voxel:
//   * its candidates are the cells of its 27-voxel neighbourhood: nine runs
//     of the voxel-sorted records, one per (dz, dy) row, each covering the
//     row's voxels x-1 .. x+1 (lanes 0..8 look up the nine runs in start[]
//     and scan their lengths);
//   * the lanes hold the candidates, 32 per chunk (up to four chunks stay in
//     registers), in the definition's order: rows (dz, dy) lexicographic,
//     voxel order inside a row;
//   * the voxel's targets are taken one at a time (their record broadcast to
//     all lanes); every lane tests its candidate against the target on the
//     hi parts (branch-free, with the margin), and the hits are appended to a
//     per-warp queue, target by target in candidate order;
//   * whenever 32 hits are queued, each lane evaluates one exact pair term and
//     a segmented reduction over the lanes sums the terms of each target (the
//     tree is fixed by the queue, so every run gives the same bits); the sums
//     enter per-target accumulators with a Kahan compensation;
//   * after up to kVoxSlots targets the batch is closed: one lane per target
//     applies AB2 and counts the next step's histograms.
// Candidate tests cost no memory access (the candidate sits in a register and
// the target is a broadcast), and the pair terms run with all 32 lanes busy
// whatever the hit pattern.  The tile's voxels need not be interior: rows
// and voxels outside the grid are empty runs.
constexpr int kVoxWarps = 8;        // warps per block
constexpr int kVoxMinBlocks = 3;    // blocks per SM (register cap of the launch bounds)
constexpr int kVoxSlots = 64;       // targets per batch
constexpr int kVoxCached = 3;       // candidate chunks kept in registers (96 candidates)
constexpr int kVoxQueue = 32 * (kVoxCached + 1);  // queued hits: < 32 left + up to 32 per cached chunk

struct VoxWarp {
    uint32_t qj[kVoxQueue];    // B position of the candidate of each queued hit
    uint32_t tq[kVoxSlots];    // B position of the target in each slot
    float acc[6][kVoxSlots];   // per slot: velocity sums x, y, z and their Kahan compensations
    uint32_t rdel[9];          // per non-empty candidate run: record index minus candidate index
    uint8_t qs[kVoxQueue];     // target slot of each queued hit
};

// Exact pair terms of the first 32 queued hits (one per lane; fewer at the end
// of a batch), summed per target slot into the accumulators; the remaining
// hits move to the front of the queue.
__device__ __noinline__ void vox_flush(const StepArgs& a, const GridDev& g, VoxWarp& w, uint32_t& qn) {
    const uint32_t lane = threadIdx.x & 31u;
    __syncwarp();
    const uint32_t cnt = min(qn, 32u);
    const bool valid = lane < cnt;
    const uint32_t sl = valid ? (uint32_t)w.qs[lane] : 0x100u + lane;  // distinct dummy slots
    float3 f = make_float3(0.f, 0.f, 0.f);
    if (valid) {
        const uint32_t j = w.qj[lane];
        const uint32_t qi = w.tq[sl];
        const float4 pi = __ldg(&a.B.rec[2 * (size_t)qi]);
        const float4 ci = __ldg(&a.B.rec[2 * (size_t)qi + 1]);
        const float4 pj = __ldg(&a.B.rec[2 * (size_t)j]);
        const float4 cj = __ldg(&a.B.rec[2 * (size_t)j + 1]);
        const float4 li = record_lo(pi, ci, g.qs);
        const float4 lj = record_lo(pj, cj, g.qs);
        pair_force(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, li.x - lj.x, li.y - lj.y, li.z - lj.z, pi.w, pj.w,
                   li.w + lj.w, ci.x, ci.y, cj.x, cj.y, affinity_f(a, record_type(ci), record_type(cj)), a.A_f,
                   a.A2m1_f, f);
    }
    // segmented suffix sums: slots are non-decreasing over the lanes, so a
    // lane adds the partial sum o lanes up whenever that lane has its slot;
    // the first lane of each slot ends with the slot's total
    const uint32_t sl_up = __shfl_up_sync(0xFFFFFFFFu, sl, 1);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float ox = __shfl_down_sync(0xFFFFFFFFu, f.x, o);
        const float oy = __shfl_down_sync(0xFFFFFFFFu, f.y, o);
        const float oz = __shfl_down_sync(0xFFFFFFFFu, f.z, o);
        const uint32_t os = __shfl_down_sync(0xFFFFFFFFu, sl, o);
        if (lane + (uint32_t)o < 32u && os == sl) {
            f.x += ox;
            f.y += oy;
            f.z += oz;
        }
    }
    if (valid && (lane == 0 || sl_up != sl)) {
        Acc3::add1(w.acc[0][sl], w.acc[3][sl], f.x);
        Acc3::add1(w.acc[1][sl], w.acc[4][sl], f.y);
        Acc3::add1(w.acc[2][sl], w.acc[5][sl], f.z);
    }
    // move the rest to the front, 32 entries at a time (sources stay ahead of
    // destinations)
    const uint32_t rest = qn - cnt;
    for (uint32_t b = 0; b < rest; b += 32u) {
        __syncwarp();
        const uint32_t k = b + lane;
        uint32_t tj = 0, ts = 0;
        if (k < rest) {
            tj = w.qj[cnt + k];
            ts = w.qs[cnt + k];
        }
        __syncwarp();
        if (k < rest) {
            w.qj[k] = tj;
            w.qs[k] = (uint8_t)ts;
        }
    }
    __syncwarp();
    qn = rest;
}

// Closes a batch: the last queued hits, then AB2 for every slot (one lane per
// target) and the next step's histograms; clears the accumulators.
template <int MODE>
__device__ __forceinline__ void vox_close(const StepArgs& a, const GridDev& g, VoxWarp& w, uint32_t& qn,
                                          uint32_t& nslot) {
    const uint32_t lane = threadIdx.x & 31u;
    while (qn) vox_flush(a, g, w, qn);
    for (uint32_t s0 = 0; s0 < nslot; s0 += 32u) {
        const uint32_t s = s0 + lane;
        const bool valid = s < nslot;
        uint32_t q = 0, nkey = 0, ntile = 0;
        if (valid) {
            q = w.tq[s];
            const float vx = __fsub_rn(w.acc[0][s], w.acc[3][s]);
            const float vy = __fsub_rn(w.acc[1][s], w.acc[4][s]);
            const float vz = __fsub_rn(w.acc[2][s], w.acc[5][s]);
            int nix, niy, niz;
            float Rf = 0.f, Rlo = 0.f;
            if (a.walls) {
                const float4 pq = __ldg(&a.B.rec[2 * (size_t)q]), cq = __ldg(&a.B.rec[2 * (size_t)q + 1]);
                Rf = pq.w;
                Rlo = record_lo(pq, cq, g.qs).w;
            }
            nkey = ab2_epilogue<MODE>(a, g, q, a_slot(a, q), vx, vy, vz, Rf, Rlo, nix, niy, niz);
            ntile = tile_index(g, nix, niy, niz, a.ltx, a.lty, a.ltz);
#pragma unroll
            for (int c = 0; c < 6; ++c) w.acc[c][s] = 0.f;
        }
        next_step_counts(a, q, nkey, ntile, valid);
    }
    __syncwarp();
    nslot = 0;
}

// Candidate runs of one voxel: run p (lane p < 9) covers the records of row
// (dz, dy) = (p / 3 - 1, p % 3 - 1) from voxel x - 1 to x + 1.  Candidate c of
// the voxel (c < L) is record c + rdel[r], r = the number of non-empty runs
// that start at or before c, minus one.
struct VoxRuns {
    uint32_t L;        // candidates
    uint32_t off;      // lane p < 9: first candidate index of run p
    uint32_t len;      // lane p < 9: its length
};

__device__ __forceinline__ uint32_t vox_cand_index(const VoxWarp& w, const VoxRuns& R, uint32_t c0) {
    const uint32_t lane = threadIdx.x & 31u;
    // bit (off_p - c0) for each non-empty run starting inside this chunk
    const bool ne = R.len != 0u;
    const uint32_t bit = (ne && R.off >= c0 && R.off < c0 + 32u) ? 1u << (R.off - c0) : 0u;
    const uint32_t starts = __reduce_or_sync(0xFFFFFFFFu, bit);
    const uint32_t before = (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, ne && R.off < c0));
    const uint32_t le = lanemask_lt() | (1u << lane);
    const uint32_t r = before + (uint32_t)__popc(starts & le) - 1u;
    return c0 + lane + w.rdel[min(r, 8u)];
}

template <int MODE>
__global__ void __launch_bounds__(kVoxWarps * 32, kVoxMinBlocks) k_force_vox(const StepArgs a) {
    __shared__ VoxWarp s_w[kVoxWarps];
    const uint32_t lane = threadIdx.x & 31u;
    VoxWarp& w = s_w[threadIdx.x >> 5];
    for (uint32_t s = lane; s < (uint32_t)kVoxSlots; s += 32u)
#pragma unroll
        for (int c = 0; c < 6; ++c) w.acc[c][s] = 0.f;
    __syncwarp();
    const float A = a.A_f;
    const uint32_t ndense = *a.ndense;
    const int TX = 1 << a.ltx, TY = 1 << a.lty, TZ = 1 << a.ltz;
    const float4 kFar = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);  // never within reach of a target
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(&a.nsparse[1], 1u);
        it = __shfl_sync(0xFFFFFFFFu, it, 0);
        if (it >= ndense) break;
        const uint32_t tile = a.tlist[it];
        const int r = rep_of_tile(a.grids, a.nrep, tile);
        const GridDev& g = a.grids[r];
        const int n0 = g.n[0], n1 = g.n[1], n2 = g.n[2];
        const uint32_t lt = tile - g.tbase;
        const uint32_t rest = lt / (uint32_t)g.nt[0];
        const int x0 = (int)(lt % (uint32_t)g.nt[0]) * TX;
        const int y0 = (int)(rest % (uint32_t)g.nt[1]) * TY;
        const int z0 = (int)(rest / (uint32_t)g.nt[1]) * TZ;
        const int x1 = min(x0 + TX, n0), y1 = min(y0 + TY, n1), z1 = min(z0 + TZ, n2);
        const float cut0 = g.qm + a.cut_eps;
        uint32_t qn = 0, nslot = 0;
        for (int vz = z0; vz < z1; ++vz)
            for (int vy = y0; vy < y1; ++vy)
                for (int vx = x0; vx < x1; ++vx) {
                    const uint32_t v =
                        g.vbase + (uint32_t)vx + (uint32_t)n0 * ((uint32_t)vy + (uint32_t)n1 * (uint32_t)vz);
                    const uint32_t t0 = a.start[v], t1 = a.start[v + 1];
                    if (t0 == t1) continue;
                    VoxRuns R;
                    uint32_t rs = 0, rl = 0;
                    if (lane < 9u) {
                        const int jz = vz + (int)(lane / 3u) - 1, jy = vy + (int)(lane % 3u) - 1;
                        if (jz >= 0 && jz < n2 && jy >= 0 && jy < n1) {
                            const uint32_t row =
                                g.vbase + (uint32_t)n0 * ((uint32_t)jy + (uint32_t)n1 * (uint32_t)jz);
                            rs = a.start[row + (uint32_t)max(vx - 1, 0)];
                            rl = a.start[row + (uint32_t)min(vx + 2, n0)] - rs;
                        }
                    }
                    uint32_t incl = rl;
#pragma unroll
                    for (int o = 1; o < 16; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += y;
                    }
                    R.L = __shfl_sync(0xFFFFFFFFu, incl, 8);
                    R.off = incl - rl;
                    R.len = rl;
                    {
                        const uint32_t nem = __ballot_sync(0xFFFFFFFFu, rl != 0u);
                        __syncwarp();
                        if (rl != 0u) w.rdel[__popc(nem & lanemask_lt())] = rs - R.off;
                        __syncwarp();
                    }
                    const uint32_t nch = (R.L + 31u) >> 5;
                    // the first chunks stay in registers; later ones are reloaded per target
                    float4 cr[kVoxCached];
                    uint32_t cjj[kVoxCached];
#pragma unroll
                    for (int k = 0; k < kVoxCached; ++k) {
                        cjj[k] = 0xFFFFFFFFu;
                        cr[k] = kFar;
                        if ((uint32_t)k < nch) {
                            const uint32_t j = vox_cand_index(w, R, 32u * (uint32_t)k);
                            if (32u * (uint32_t)k + lane < R.L) {
                                cjj[k] = j;
                                cr[k] = __ldg(&a.B.rec[2 * (size_t)j]);
                            }
                        }
                    }
                    for (uint32_t tb = t0; tb < t1;) {
                        const uint32_t take = min(t1 - tb, (uint32_t)kVoxSlots - nslot);
                        if (take == 0) {
                            vox_close<MODE>(a, g, w, qn, nslot);
                            continue;
                        }
                        for (uint32_t k = lane; k < take; k += 32u) w.tq[nslot + k] = tb + k;
                        __syncwarp();
                        for (uint32_t k = 0; k < take; ++k) {
                            const uint32_t q = tb + k;
                            const uint32_t slot = nslot + k;
                            const float4 pi = __ldg(&a.B.rec[2 * (size_t)q]);
                            const float cut_i = fmaf(A, pi.w, cut0);
                            // test: append the hits of one chunk to the queue (candidate order)
                            auto test = [&](const float4& c4, uint32_t j) {
                                const bool hit = j != q && candidate_hit(pi.x - c4.x, pi.y - c4.y, pi.z - c4.z, A,
                                                                         c4.w, cut_i);
                                const uint32_t m = __ballot_sync(0xFFFFFFFFu, hit);
                                if (hit) {
                                    const uint32_t pos = qn + (uint32_t)__popc(m & lanemask_lt());
                                    w.qj[pos] = j;
                                    w.qs[pos] = (uint8_t)slot;
                                }
                                qn += (uint32_t)__popc(m);
                            };
#pragma unroll
                            for (int ch = 0; ch < kVoxCached; ++ch)
                                if ((uint32_t)ch < nch) test(cr[ch], cjj[ch]);
                            while (qn >= 32u) vox_flush(a, g, w, qn);
                            for (uint32_t ch = kVoxCached; ch < nch; ++ch) {
                                const uint32_t j = vox_cand_index(w, R, 32u * ch);
                                const bool in = 32u * ch + lane < R.L;
                                test(in ? __ldg(&a.B.rec[2 * (size_t)j]) : kFar, in ? j : 0xFFFFFFFFu);
                                if (qn >= 32u) vox_flush(a, g, w, qn);
                            }
                        }
                        nslot += take;
                        tb += take;
                    }
                }
        vox_close<MODE>(a, g, w, qn, nslot);
    }
}

// ------------------------------------------------------ sparse list ----
// After the tile kernel (which may hand tiles back): B position and voxel key
// of every cell whose tile is not dense, in runs of a warp's 32 consecutive
// cells, and whether the cell is alone in its voxel (its sorted neighbours
// q - 1 and q + 1 have other keys).
// A block takes 4 x 256 cells per round, each thread 4 cells 256 apart, so the
// loads of a round (keys, then tile flags) are issued together: the kernel
// waits on memory, and a thread's rounds are sequential.  One atomic per
// round reserves the block's list entries (one counter serves the whole grid).
constexpr int kListBlock = 256, kListPer = 4;

__global__ void __launch_bounds__(kListBlock) k_sparse_list(const StepArgs a) {
    __shared__ uint32_t s_cnt[kListPer][kListBlock / 32];
    __shared__ uint32_t s_base;
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    constexpr uint32_t kNone = 0xFFFFFFFFu;  // above every voxel key
    constexpr uint32_t kRound = kListBlock * kListPer;
    for (uint32_t base = blockIdx.x * kRound; base < a.n; base += gridDim.x * kRound) {
        uint32_t k[kListPer], kp[kListPer], kn[kListPer];
        bool sparse[kListPer];
#pragma unroll
        for (int j = 0; j < kListPer; ++j) {
            const uint32_t q = base + (uint32_t)j * kListBlock + threadIdx.x;
            const bool last = lane == 31u || q + 1u >= a.n;  // next cell not in this warp's registers
            k[j] = q < a.n ? a.vkey_s[q] : 0u;
            kp[j] = (lane == 0u && q > 0u && q < a.n) ? a.vkey_s[q - 1u] : kNone;
            kn[j] = (last && q + 1u < a.n) ? a.vkey_s[q + 1u] : kNone;
        }
#pragma unroll
        for (int j = 0; j < kListPer; ++j) {
            const uint32_t q = base + (uint32_t)j * kListBlock + threadIdx.x;
            sparse[j] = false;
            if (q < a.n) {
                const int r = rep_of_cell(a.grids, a.nrep, q);
                const GridDev& g = a.grids[r];
                const Cell3 c = decode(k[j], g);
                sparse[j] = !a.tdense[tile_index(g, c.ix, c.iy, c.iz, a.ltx, a.lty, a.ltz)];
            }
        }
        uint32_t m[kListPer];
#pragma unroll
        for (int j = 0; j < kListPer; ++j) {
            const uint32_t q = base + (uint32_t)j * kListBlock + threadIdx.x;
            const uint32_t up = __shfl_up_sync(0xFFFFFFFFu, k[j], 1);
            const uint32_t dn = __shfl_down_sync(0xFFFFFFFFu, k[j], 1);
            if (lane != 0u) kp[j] = up;
            if (!(lane == 31u || q + 1u >= a.n)) kn[j] = dn;
            m[j] = __ballot_sync(0xFFFFFFFFu, sparse[j]);
            if (lane == 0u) s_cnt[j][wib] = (uint32_t)__popc(m[j]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // offsets of the (round part, warp) groups, and the block's reservation
            uint32_t t = 0;
            for (int j = 0; j < kListPer; ++j)
                for (int w = 0; w < kListBlock / 32; ++w) {
                    const uint32_t c = s_cnt[j][w];
                    s_cnt[j][w] = t;
                    t += c;
                }
            s_base = t ? atomicAdd(a.nsparse, t) : 0u;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kListPer; ++j)
            if (sparse[j]) {
                const uint32_t q = base + (uint32_t)j * kListBlock + threadIdx.x;
                const uint32_t alone = (kp[j] != k[j] && kn[j] != k[j]) ? 0x80000000u : 0u;
                a.slist[s_base + s_cnt[j][wib] + __popc(m[j] & lanemask_lt())] = make_uint2(q | alone, k[j]);
            }
        __syncthreads();  // s_cnt and s_base are rewritten by the next round
    }
}

// --------------------------------------------------------- tile kernel ----
// One CTA per dense tile of 4 x 4 x 4 voxels, per tile:
//   1. halo row table: for each (y, z) row of the halo (one voxel around the
//      tile), the global start of its run of force records and the voxel
//      boundaries inside it;
//   2. TMA: one bulk copy per row (its 32-byte records are contiguous) into
//      shared memory, completion on an mbarrier (bounded wait);
//   3. for every core voxel, the shared-memory indices of its 27-voxel
//      neighbourhood (9 contiguous row ranges) are written into one list;
//   4. one thread per target cell scans its voxel's list in blocks of 32
//      candidates: a branch-free cutoff test on the hi parts builds a hit
//      mask per block, then the exact pair terms of the hits are summed in
//      list order; then AB2 and the next-step histograms.
// A tile whose halo or lists do not fit clears its dense flag and leaves its
// cells to the thread-per-cell kernel, which runs after this one.

// Exclusive scan of v[0..n) in place by one warp (n small); returns the total.
__device__ __forceinline__ uint32_t warp_scan_inplace(uint32_t* v, int n) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t carry = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + (int)lane;
        const uint32_t x = i < n ? v[i] : 0u;
        uint32_t inc = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, inc, o);
            if ((int)lane >= o) inc += y;
        }
        if (i < n) v[i] = carry + inc - x;
        carry += __shfl_sync(0xFFFFFFFFu, inc, 31);
    }
    return carry;
}

// Tile of TX x 4 x TZ voxels (TX = 2^LX, TZ = 2^LZ; 4x4x4, 4x4x8 or 8x4x4):
// threads per CTA (about one per target), CTAs per SM, staged halo records (a
// dense core 4x4x4 tile holds ~490 of its 216 halo voxels) and candidate-list
// entries per tile.
template <int LX, int LZ>
struct TileCfg {
    static constexpr int TX = 1 << LX, TZ = 1 << LZ, NV = 4 * TX * TZ;
    static constexpr int TT = NV <= 64 ? 160 : 320;
    static constexpr int MINB = NV <= 64 ? 6 : 3;
    static constexpr int CAP = NV <= 64 ? 640 : 1088;
    static constexpr int LCAP = NV <= 64 ? 5120 : 10240;
    static constexpr size_t DYN = (size_t)CAP * 2 * sizeof(float4) + (size_t)LCAP * 2;
};

template <int MODE, int LX, int LZ>
__global__ void __launch_bounds__(TileCfg<LX, LZ>::TT, TileCfg<LX, LZ>::MINB) k_force_tile(const StepArgs a) {
    using C = TileCfg<LX, LZ>;
    constexpr int kTT = C::TT, kTCap = C::CAP, kTListCap = C::LCAP, TX = C::TX, TZ = C::TZ;
    // halo rows run along x: RL voxels each, HY x HZ of them
    constexpr int RL = TX + 2, HY = 6, HZ = TZ + 2, NB = RL + 1, NROW = HY * HZ, NVOX = C::NV;
    static_assert(NROW <= 64 && 64 + NVOX <= kTT, "thread roles of the set-up phase");
    extern __shared__ __align__(128) unsigned char dsm[];
    float4* srec = reinterpret_cast<float4*>(dsm);        // staged force records (two float4 each)
    uint16_t* clist = reinterpret_cast<uint16_t*>(srec + 2 * kTCap);   // per-voxel candidate lists
    __shared__ uint32_t s_row_gs[NROW];
    __shared__ uint32_t s_row_off[NROW + 1];
    __shared__ uint32_t s_row_vb[NROW][NB];
    __shared__ uint32_t s_vox_loff[NVOX + 1];   // list offset of each core voxel
    __shared__ uint32_t s_vox_toff[NVOX + 1];   // first target number of each core voxel
    __shared__ uint16_t s_vp_off[NVOX][9];      // offset of each neighbour row inside a voxel's list
    __shared__ uint8_t s_tvox[kTCap];           // core voxel of each target (< 128)
    __shared__ int s_flag;                       // copy timeout
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_next;                  // next tile claimed by this CTA

    const int tid = threadIdx.x;
    const uint32_t lane = tid & 31u;
    const int warp = tid >> 5;
    const float A = a.A_f;
    if (tid == 0) {
        s_flag = 0;
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t ndense = *a.ndense;
    // tiles are claimed one at a time from a cursor (their cost varies with
    // their cell count), the claim's barrier also ending the previous tile:
    // its shared tables and records are reused by the next one
    auto claim = [&]() -> uint32_t {
        if (tid == 0) s_next = atomicAdd(&a.nsparse[1], 1u);
        __syncthreads();
        return s_next;
    };
    for (uint32_t it = claim(); it < ndense; it = claim()) {
        const uint32_t tile = a.tlist[it];
        const int r = rep_of_tile(a.grids, a.nrep, tile);
        const GridDev& g = a.grids[r];
        const uint32_t lt = tile - g.tbase;
        const int bx = (int)(lt % (uint32_t)g.nt[0]);
        const uint32_t rest = lt / (uint32_t)g.nt[0];
        const int by = (int)(rest % (uint32_t)g.nt[1]);
        const int bz = (int)(rest / (uint32_t)g.nt[1]);
        const int x_lo = TX * bx - 1, y_lo = 4 * by - 1, z_lo = TZ * bz - 1;
        // 1. halo row table: row rr = (y - y_lo) + 6 (z - z_lo); boundary k of a
        // row is the start of its voxel x_lo + k (k = RL: the end of the row)
        for (int w = tid; w < NROW * NB; w += kTT) {
            const int rr = w / NB, k = w - rr * NB;
            const int yy = y_lo + rr % HY, zz = z_lo + rr / HY;
            const uint32_t rowv = g.vbase + (uint32_t)g.n[0] * ((uint32_t)yy + (uint32_t)g.n[1] * (uint32_t)zz);
            s_row_vb[rr][k] = a.start[rowv + (uint32_t)(x_lo + k)];
        }
        __syncthreads();
        if (warp == 0) {
            for (int rr = (int)lane; rr < NROW; rr += 32) {
                const uint32_t gs = s_row_vb[rr][0];
                s_row_gs[rr] = gs;
                s_row_off[rr] = s_row_vb[rr][RL] - gs;  // row length, scanned below
            }
            __syncwarp();
            const uint32_t total = warp_scan_inplace(s_row_off, NROW);
            if (lane == 0) s_row_off[NROW] = total;
        }
        __syncthreads();
        for (int w = tid; w < NROW * NB; w += kTT) {
            const int rr = w / NB, k = w - rr * NB;
            s_row_vb[rr][k] -= s_row_gs[rr];  // boundaries relative to the row start
        }
        const uint32_t total = s_row_off[NROW];
        __syncthreads();
        if (total > (uint32_t)kTCap) {  // does not fit: leave the tile to the thread-per-cell kernel
            if (tid == 0) a.tdense[tile] = 0;
            continue;
        }
        // 2. TMA bulk copies of the halo rows, one row per thread; the barrier
        // expects the bytes of all rows (its single arrival comes with them)
        if (tid < NROW) {
            const int rr = tid;
            const uint32_t len = s_row_vb[rr][RL];
            fence_proxy_async();
            if (tid == 0)
                mbar_arrive_expect_tx(&s_bar, total * 2u * (uint32_t)sizeof(float4) +
                                                  ((a.fault & kFaultTileWait) ? 16u : 0u));
            if (len)
                bulk_g2s(&srec[2 * s_row_off[rr]], &a.B.rec[2 * (size_t)s_row_gs[rr]],
                         len * 2u * (uint32_t)sizeof(float4), &s_bar);
        } else if (tid >= 64 && tid < 64 + NVOX) {
            // 3a (overlaps the copies). per-voxel list lengths, neighbour-row offsets, target counts
            const int v = tid - 64;
            const int cx = v & (TX - 1), cy = (v >> LX) & 3, cz = v >> (LX + 2);
            uint32_t len = 0;
            int p = 0;
#pragma unroll
            for (int dz = 0; dz < 3; ++dz)
#pragma unroll
                for (int dy = 0; dy < 3; ++dy, ++p) {
                    const int r2 = (cy + dy) + HY * (cz + dz);
                    s_vp_off[v][p] = (uint16_t)len;
                    len += s_row_vb[r2][cx + 3] - s_row_vb[r2][cx];
                }
            const int rr = (cy + 1) + HY * (cz + 1);
            s_vox_loff[v] = len;
            s_vox_toff[v] = s_row_vb[rr][cx + 2] - s_row_vb[rr][cx + 1];
        }
        __syncthreads();
        if (warp == 0) {
            const uint32_t l_total = warp_scan_inplace(s_vox_loff, NVOX);
            const uint32_t t_total = warp_scan_inplace(s_vox_toff, NVOX);
            if (lane == 0) {
                s_vox_loff[NVOX] = l_total;
                s_vox_toff[NVOX] = t_total;
            }
        }
        // 2b. wait for the halo
        if (!mbar_wait_bounded(&s_bar, phase, a.wait_ns)) s_flag = 1;
        phase ^= 1u;
        __syncthreads();
        if (s_flag) {
            if (tid == 0) atomicOr(a.err, kErrTimeout);
            mbar_wait_bounded(&s_bar, phase ^ 1u, a.wait_ns);  // let copies in flight land first
            return;
        }
        if (s_vox_loff[NVOX] > (uint32_t)kTListCap) {  // lists do not fit: same hand-back
            if (tid == 0) a.tdense[tile] = 0;
            __syncthreads();
            continue;
        }
        // 3b. candidate index lists, one (voxel, neighbour row) pair per thread,
        // and the core voxel of every target
        for (int w = tid; w < NVOX * 9; w += kTT) {
            const int v = w / 9, p = w - v * 9;
            const int cx = v & (TX - 1), cy = (v >> LX) & 3, cz = v >> (LX + 2);
            const int r2 = (cy + p % 3) + HY * (cz + p / 3);
            uint32_t o = s_vox_loff[v] + s_vp_off[v][p];
            const uint32_t j1 = s_row_off[r2] + s_row_vb[r2][cx + 3];
            for (uint32_t j = s_row_off[r2] + s_row_vb[r2][cx]; j < j1; ++j) clist[o++] = (uint16_t)j;
            if (p == 0)
                for (uint32_t t = s_vox_toff[v]; t < s_vox_toff[v + 1]; ++t) s_tvox[t] = (uint8_t)v;
        }
        __syncthreads();
        // 4. one thread per target; in a warp pass with g <= 16 targets (the
        // last pass of a tile) each target's candidate list is split into L
        // contiguous parts (L lanes per target, L g <= 32) whose Kahan sums
        // are combined by a fixed tree, so the pass costs a fraction of a
        // full one instead of the work of its busiest target
        const uint32_t T = s_vox_toff[NVOX];
        for (uint32_t t0 = (uint32_t)warp * 32u; t0 < T; t0 += kTT) {
            const uint32_t gcnt = min(32u, T - t0);
            const uint32_t lsh = gcnt > 16u ? 0u : gcnt > 8u ? 1u : gcnt > 4u ? 2u : gcnt > 2u ? 3u : gcnt > 1u ? 4u : 5u;
            const uint32_t L = 1u << lsh;
            const uint32_t part = lane & (L - 1u);
            const uint32_t t = t0 + (lane >> lsh);
            const bool valid = (lane >> lsh) < gcnt;
            uint32_t nkey = 0, ntile = 0, q = 0, src = 0;
            float Ri = 0.f, Rlo_i = 0.f;
            Acc3 acc;
            acc.zero();
            if (valid) {
                const int v = s_tvox[t];
                const uint32_t k = t - s_vox_toff[v];
                const int cx = v & (TX - 1), cy = (v >> LX) & 3, cz = v >> (LX + 2);
                const int rr = (cy + 1) + HY * (cz + 1);
                const uint32_t in_row = s_row_vb[rr][cx + 1] + k;
                q = s_row_gs[rr] + in_row;
                if (part == 0u) src = a_slot(a, q);  // its state, read after the scan
                const uint32_t si = s_row_off[rr] + in_row;
                const float4 pi = srec[2 * si];
                const float4 qi = srec[2 * si + 1];
                const float4 li = record_lo(pi, qi, g.qs);
                Ri = pi.w;
                Rlo_i = li.w;
                const float cut_i = fmaf(A, pi.w, g.qm + a.cut_eps);
                // this lane's part [p0, p1) of the voxel's list, scanned in blocks
                // of 32 candidates (up to three blocks at a time): a branch-free
                // test on the hi parts builds one hit mask per block, then the
                // exact pair terms of all hits (from hi + lo) are summed in list
                // order in a single loop, so a warp's divergent iterations are
                // its largest total hit count, not a sum of per-block maxima
                const uint32_t l0 = s_vox_loff[v], len = s_vox_loff[v + 1] - l0;
                const uint32_t p0 = l0 + ((len * part) >> lsh), l1 = l0 + ((len * (part + 1u)) >> lsh);
                for (uint32_t cb = p0; cb < l1; cb += 96u) {
                    uint32_t m[3] = {0u, 0u, 0u};
#pragma unroll
                    for (int b = 0; b < 3; ++b) {
                        const uint32_t c0 = cb + 32u * (uint32_t)b;
                        const uint32_t nc = c0 < l1 ? min(32u, l1 - c0) : 0u;
#pragma unroll 8
                        for (uint32_t k2 = 0; k2 < nc; ++k2) {
                            const float4 pj = srec[2 * (uint32_t)clist[c0 + k2]];
                            m[b] |= (candidate_hit(pi.x - pj.x, pi.y - pj.y, pi.z - pj.z, A, pj.w, cut_i) ? 1u : 0u)
                                    << k2;
                        }
                    }
                    // the hit loop, specialised on the affinity table (without
                    // one, the factor is the literal 1 and costs nothing)
                    auto hits = [&](auto with_affinity) {
                        constexpr bool kAff = decltype(with_affinity)::value;
                        while (m[0] | m[1] | m[2]) {
                            const int b = m[0] ? 0 : (m[1] ? 1 : 2);
                            const uint32_t mb = b == 0 ? m[0] : (b == 1 ? m[1] : m[2]);
                            const uint32_t k2 = (uint32_t)(__ffs(mb) - 1);
                            const uint32_t rest = mb & (mb - 1u);
                            if (b == 0) m[0] = rest; else if (b == 1) m[1] = rest; else m[2] = rest;
                            const uint32_t jj = clist[cb + 32u * (uint32_t)b + k2];
                            const float4 p2 = srec[2 * jj];
                            const float4 q2 = srec[2 * jj + 1];
                            const float4 l2 = record_lo(p2, q2, g.qs);
                            const float aij =
                                kAff ? __ldg(&a.aff_f[record_type(qi) * kMaxTypes + record_type(q2)]) : 1.0f;
                            pair_term(pi.x - p2.x, pi.y - p2.y, pi.z - p2.z, li.x - l2.x, li.y - l2.y,
                                      li.z - l2.z, pi.w, p2.w, li.w + l2.w, qi.x, qi.y, q2.x, q2.y, aij, A,
                                      a.A2m1_f, acc);
                        }
                    };
                    if (a.ntypes > 0)
                        hits(std::true_type{});
                    else
                        hits(std::false_type{});
                }
            }
            // the parts of a target: lane part + o's sum into lane part, for
            // part a multiple of 2 o (all lanes take part in the shuffles)
            for (uint32_t o = 1u; o < L; o <<= 1) {
                const float ox = __shfl_down_sync(0xFFFFFFFFu, acc.x, o);
                const float oy = __shfl_down_sync(0xFFFFFFFFu, acc.y, o);
                const float oz = __shfl_down_sync(0xFFFFFFFFu, acc.z, o);
                const float ocx = __shfl_down_sync(0xFFFFFFFFu, acc.cx, o);
                const float ocy = __shfl_down_sync(0xFFFFFFFFu, acc.cy, o);
                const float ocz = __shfl_down_sync(0xFFFFFFFFu, acc.cz, o);
                if ((part & (2u * o - 1u)) == 0u) {
                    acc.add(ox, oy, oz);
                    acc.add(-ocx, -ocy, -ocz);
                }
            }
            const bool owner = valid && part == 0u;
            if (owner) {
                int nix, niy, niz;
                nkey = ab2_epilogue<MODE>(a, g, q, src, acc.vx(), acc.vy(), acc.vz(), Ri, Rlo_i, nix, niy, niz);
                ntile = tile_index(g, nix, niy, niz, a.ltx, a.lty, a.ltz);
            }
            next_step_counts(a, q, nkey, ntile, owner);
        }
    }
}

// ---------------------------------------------------------------- FP64 ----
// All-FP64 mode.  An FP32 test with a relative margin of 1e-4 on the squared
// cutoff discards candidates that are certainly out of range; the survivors
// are evaluated in FP64 from the FP64 positions and parameters with the same
// operations, in the same order, as the definition (no contraction, IEEE sqrt
// and division), and summed in the definition's candidate order.
__global__ void __launch_bounds__(kCellBlock) k_force_fp64(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const float A = a.A_f;
    const double Ad = a.A_d;
    const size_t np = a.npad;
    for (uint32_t base = warp * 32u; base < a.n; base += nwarps * 32u) {
        const uint32_t q = base + lane;
        const bool valid = q < a.n;
        uint32_t nkey = 0, ntile = 0;
        if (valid) {
            const int r = rep_of_cell(a.grids, a.nrep, q);
            const GridDev& g = a.grids[r];
            const Cell3 c = decode(a.vkey_s[q], g);
            const float4 pi = a.B.rec[2 * (size_t)q];
            const uint32_t src = a.perm[q];
            const uint32_t idi = a.A.id[src];
            const double xi = a.A.pos64[src], yi = a.A.pos64[np + src], zi = a.A.pos64[2 * np + src];
            const double Ri = a.R64[idi], ccri = a.ccr64[idi], ccai = a.cca64[idi];
            const uint32_t ti = a.ntypes > 0 ? record_type(a.B.rec[2 * (size_t)q + 1]) : 0u;
            const float cut_i = fmaf(A, pi.w, g.qm + a.cut_eps);
            double ax = 0.0, ay = 0.0, az = 0.0;
            for (int dz = -1; dz <= 1; ++dz) {
                const int jz = c.iz + dz;
                if (jz < 0 || jz >= g.n[2]) continue;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int jy = c.iy + dy;
                    if (jy < 0 || jy >= g.n[1]) continue;
                    const uint32_t row = g.vbase + (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
                    const int jx0 = c.ix > 0 ? c.ix - 1 : 0;
                    const int jx1 = c.ix + 1 < g.n[0] ? c.ix + 1 : g.n[0] - 1;
                    uint32_t s = a.start[row + jx0];
                    for (int jx = jx0; jx <= jx1; ++jx) {
                        const uint32_t e = a.start[row + jx + 1];
                        for (uint32_t j = s; j < e; ++j) {
                            if (j == q) continue;
                            const float4 pj = a.B.rec[2 * (size_t)j];
                            const float rx = pi.x - pj.x, ry = pi.y - pj.y, rz = pi.z - pj.z;
                            const float d2f = rx * rx + ry * ry + rz * rz;
                            const float cut = fmaf(A, pj.w, cut_i);
                            if (!(d2f <= cut * cut * 1.0001f + 1e-2f)) continue;
                            const uint32_t sj = a.perm[j];
                            const uint32_t idj = a.A.id[sj];
                            const double dx = __dsub_rn(xi, a.A.pos64[sj]);
                            const double dy2 = __dsub_rn(yi, a.A.pos64[np + sj]);
                            const double dz2 = __dsub_rn(zi, a.A.pos64[2 * np + sj]);
                            const double dd2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2)),
                                                         __dmul_rn(dz2, dz2));
                            const double d = __dsqrt_rn(dd2);
                            if (!(d > 0.0)) continue;
                            const double S = __dadd_rn(Ri, a.R64[idj]);
                            const double AS = __dmul_rn(Ad, S);
                            if (!(d < AS)) continue;
                            double cf = 0.0;
                            if (d < S) {
                                const double t = __dsub_rn(1.0, __ddiv_rn(d, S));
                                cf = __dmul_rn(__dsqrt_rn(__dmul_rn(ccri, a.ccr64[idj])), __dmul_rn(t, t));
                            }
                            const double ta = __dsub_rn(1.0, __ddiv_rn(d, AS));
                            // adhesion coefficient (a_ij sqrt(cca_i cca_j)); a_ij = 1 without affinity
                            const double aij =
                                a.ntypes > 0 ? a.aff_d[ti * kMaxTypes + record_type(a.B.rec[2 * (size_t)j + 1])] : 1.0;
                            cf = __dsub_rn(cf, __dmul_rn(__dmul_rn(aij, __dsqrt_rn(__dmul_rn(ccai, a.cca64[idj]))),
                                                         __dmul_rn(ta, ta)));
                            const double sc = __ddiv_rn(cf, d);
                            ax = __dadd_rn(ax, __dmul_rn(sc, dx));
                            ay = __dadd_rn(ay, __dmul_rn(sc, dy2));
                            az = __dadd_rn(az, __dmul_rn(sc, dz2));
                        }
                        s = e;
                    }
                }
            }
            double v[3] = {ax, ay, az};
            const double xo[3] = {xi, yi, zi};
            if (a.walls) wall_terms(a, g, xo, Ri, v);  // after the pair terms, as the definition orders them
            double xn[3];
            bool finite = true;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double vp = a.A.vp64[d * np + src];
                if (a.integrate) {
                    const double inc = __dmul_rn(a.dt_d, __dsub_rn(__dmul_rn(1.5, v[d]), __dmul_rn(0.5, vp)));
                    xn[d] = __dadd_rn(xo[d], inc);
                } else {
                    xn[d] = xo[d];
                }
                a.B.pos64[d * np + q] = xn[d];
                a.B.vp64[d * np + q] = a.integrate ? v[d] : vp;
                if (!a.integrate) a.vout_d[d * np + q] = v[d];
                finite = finite && isfinite(xn[d]) && isfinite(v[d]);
            }
            if (!finite) atomicOr(a.err, kErrNonFinite);
            const int ix = axis_index_f64(xn[0], g.lo[0], g.inv_h, g.n[0]);
            const int iy = axis_index_f64(xn[1], g.lo[1], g.inv_h, g.n[1]);
            const int iz = axis_index_f64(xn[2], g.lo[2], g.inv_h, g.n[2]);
            nkey = g.vbase + (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy + (uint32_t)g.n[1] * (uint32_t)iz);
            ntile = tile_index(g, ix, iy, iz, a.ltx, a.lty, a.ltz);
        }
        next_step_counts(a, q, nkey, ntile, valid);
    }
}

// ------------------------------------------------------ pair stats ----
// One thread per cell of the voxel order in B: counts its candidates (cells of
// the 27 neighbour voxels, itself excluded) and its interacting neighbours,
// decided in FP64 from caller-order positions exactly as the definition does.
__global__ void __launch_bounds__(kCellBlock) k_pair_stats(const StepArgs a, const double* __restrict__ xyz,
                                                          unsigned long long* __restrict__ out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    unsigned long long cand = 0, hits = 0;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const int r = rep_of_cell(a.grids, a.nrep, q);
        const GridDev& g = a.grids[r];
        const Cell3 c = decode(a.vkey_s[q], g);
        const uint32_t idi = a.B.id[q];
        const double xi = xyz[3 * (size_t)idi], yi = xyz[3 * (size_t)idi + 1], zi = xyz[3 * (size_t)idi + 2];
        const double Ri = a.R64[idi];
        for (int dz = -1; dz <= 1; ++dz) {
            const int jz = c.iz + dz;
            if (jz < 0 || jz >= g.n[2]) continue;
            for (int dy = -1; dy <= 1; ++dy) {
                const int jy = c.iy + dy;
                if (jy < 0 || jy >= g.n[1]) continue;
                const uint32_t row = g.vbase + (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
                const int jx0 = c.ix > 0 ? c.ix - 1 : 0;
                const int jx1 = c.ix + 1 < g.n[0] ? c.ix + 1 : g.n[0] - 1;
                const uint32_t s = a.start[row + jx0], e = a.start[row + jx1 + 1];
                for (uint32_t j = s; j < e; ++j) {
                    if (j == q) continue;
                    ++cand;
                    const uint32_t idj = a.B.id[j];
                    const double dx = __dsub_rn(xi, xyz[3 * (size_t)idj]);
                    const double dy2 = __dsub_rn(yi, xyz[3 * (size_t)idj + 1]);
                    const double dz2 = __dsub_rn(zi, xyz[3 * (size_t)idj + 2]);
                    const double d = __dsqrt_rn(
                        __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy2, dy2)), __dmul_rn(dz2, dz2)));
                    if (d > 0.0 && d < __dmul_rn(a.A_d, __dadd_rn(Ri, a.R64[idj]))) ++hits;
                }
            }
        }
    }
    // warp sums, one atomic per warp and counter
    for (int o = 16; o > 0; o >>= 1) {
        cand += __shfl_down_sync(0xFFFFFFFFu, cand, o);
        hits += __shfl_down_sync(0xFFFFFFFFu, hits, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicAdd(&out[0], cand);
        atomicAdd(&out[1], hits);
    }
}

// ---- tile kernel launch ----
template <int MODE, int LX, int LZ>
cudaError_t launch_tile_mode(const StepArgs& a, int grid, cudaStream_t s) {
    using C = TileCfg<LX, LZ>;
    // the dynamic shared-memory limit is a per-device function attribute: set
    // it once for each device this process launches on (devices 0..63)
    static std::atomic<unsigned long long> configured{0ull};
    auto k = k_force_tile<MODE, LX, LZ>;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(configured.load() & bit)) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::DYN);
        if (e != cudaSuccess) return e;
        configured.fetch_or(bit);
    }
    k<<<grid, C::TT, C::DYN, s>>>(a);
    return cudaGetLastError();
}

template <int MODE>
cudaError_t launch_vox_mode(const StepArgs& a, int grid, cudaStream_t s) {
    k_force_vox<MODE><<<grid, kVoxWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

template <int LX, int LZ>
int tile_grid_for(int sms) {
    using C = TileCfg<LX, LZ>;
    int nb = 0;
    cudaFuncSetAttribute(k_force_tile<kMixedKahan, LX, LZ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)C::DYN);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_tile<kMixedKahan, LX, LZ>, C::TT, C::DYN);
    return sms * (nb > 0 ? nb : 1);
}

template <int MODE>
cudaError_t launch_tile_shape(const StepArgs& a, int grid, cudaStream_t s) {
    if (a.ltx == 3) return launch_tile_mode<MODE, 3, 2>(a, grid, s);
    if (a.ltz == 3) return launch_tile_mode<MODE, 2, 3>(a, grid, s);
    return launch_tile_mode<MODE, 2, 2>(a, grid, s);
}

}  // namespace

bool tile_shape_supported(int ltx, int lty, int ltz) {
    return lty == 2 && ((ltx == 2 && (ltz == 2 || ltz == 3)) || (ltx == 3 && ltz == 2));
}

int force_max_blocks_per_sm(int mode, int block) {
    int nb = 0;
    if (mode == kFP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_fp64, block, 0);
    else if (mode == kMixedFP64Pos)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_cells<kMixedFP64Pos, false>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_cells<kMixedKahan, false>, block, 0);
    return nb > 0 ? nb : 1;
}

int tile_kernel_grid(const StepArgs& a, int sms) {
    if (a.tile_kernel == kTileKernelVox) {
        int nb = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_vox<kMixedKahan>, kVoxWarps * 32, 0);
        return sms * (nb > 0 ? nb : 1);
    }
    if (a.ltx == 3) return tile_grid_for<3, 2>(sms);
    return a.ltz == 3 ? tile_grid_for<2, 3>(sms) : tile_grid_for<2, 2>(sms);
}

cudaError_t launch_tile_classify(const StepArgs& a, cudaStream_t s) {
    if (a.ntiles == 0) return cudaSuccess;
    int g = (int)((a.ntiles + 255u) / 256u);
    g = std::min(g, device_sms() * 16);
    k_tile_classify<<<g, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_force_tiles(const StepArgs& a, int grid, cudaStream_t s) {
    if (a.n == 0 || !a.use_tiles || a.mode == kFP64) return cudaSuccess;
    if (a.tile_kernel == kTileKernelVox)
        return a.mode == kMixedFP64Pos ? launch_vox_mode<kMixedFP64Pos>(a, grid, s)
                                       : launch_vox_mode<kMixedKahan>(a, grid, s);
    if (a.mode == kMixedFP64Pos) return launch_tile_shape<kMixedFP64Pos>(a, grid, s);
    return launch_tile_shape<kMixedKahan>(a, grid, s);
}

cudaError_t launch_sparse_list(const StepArgs& a, int grid, cudaStream_t s) {
    if (a.n == 0 || !a.use_tiles || a.mode == kFP64) return cudaSuccess;
    k_sparse_list<<<grid, kListBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_pair_stats(const StepArgs& a, const double* xyz, unsigned long long* out, int grid,
                              cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_pair_stats<<<grid, kCellBlock, 0, s>>>(a, xyz, out);
    return cudaGetLastError();
}

cudaError_t launch_force_cells(const StepArgs& a, int grid, int block, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.mode == kFP64)
        k_force_fp64<<<grid, block, 0, s>>>(a);
    else if (a.mode == kMixedFP64Pos && a.ntypes > 0)
        k_force_cells<kMixedFP64Pos, true><<<grid, block, 0, s>>>(a);
    else if (a.mode == kMixedFP64Pos)
        k_force_cells<kMixedFP64Pos, false><<<grid, block, 0, s>>>(a);
    else if (a.ntypes > 0)
        k_force_cells<kMixedKahan, true><<<grid, block, 0, s>>>(a);
    else
        k_force_cells<kMixedKahan, false><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mk
