// Internal declarations of libmech: device data layout, kernel argument
// block and the launch wrappers of each translation unit.
//
// Data layout in HBM (one handle, n cells, V voxels over all replicates):
//   * per-cell state, double-buffered (A = current order, B = the voxel order
//     built this step), SoA with stride `npad` per component:
//       pos64  [3][npad] double   positions (FP64 and FP64-position modes)
//       posf   [3][npad] float    positions x_hi (Kahan mode)
//       comp   [3][npad] float    Kahan compensation c, value = x_hi - c
//       vp64   [3][npad] double   previous velocity (FP64 mode)
//       vpf    [3][npad] float    previous velocity (mixed modes)
//       id     [n]       u32      caller index of the cell
//       rec    [2n]      float4   force record of cell i, 32 contiguous bytes:
//                                 rec[2i]   = {x_hi, y_hi, z_hi, R}: position
//                                 relative to the replicate's grid centre as a
//                                 hi part on a power-of-two grid q, and the
//                                 radius (FP32);
//                                 rec[2i+1] = {sqrt(ccr), sqrt(cca), lo_xy,
//                                 lo_zr}: the coefficient square roots, then
//                                 three 16-bit fixed-point residuals x_lo,
//                                 y_lo, z_lo in units of q / 2^15, then
//                                 R - (float)R in units of ulp(R) / 2^11
//                                 (12 bits) and the cell type (4 bits, the
//                                 top of lo_zr)
//     The canonicalisation pass writes only the force records in B order;
//     the force kernels read each cell's state (positions, compensation,
//     previous velocity) in A order at perm[q] (nearly sequential: cells that
//     stay in their voxel keep their relative order) and write its new state
//     at q in B order.
//   * binning scratch: key [n] (next voxel of each cell in A order), vkey_s
//     [n] (key in B order), perm [n] (A index of the cell at each B
//     position), tmp [n] u64 (id << 32 | A index, scattered by key),
//     count[2][Vpad] (histograms of this and the next step; the scatter
//     counts this step's histogram back down to zero), start[Vpad] (exclusive
//     scan of count: cells of voxel v are the sorted positions start[v] ..
//     start[v+1]-1), occ[Vpad/32 + 1] (bit v: count > 0), bcount[2][Vpad /
//     8192] (cells of each scan block of 8,192 voxels, counted with the
//     histograms, so a step's scan starts from the block sums).
//   * voxel tiles: the grid is cut into blocks of TX x TY x TZ voxels (powers
//     of two); tcount[2][T] counts the cells of each tile (this step, next
//     step), tdense[T] flags the tiles processed by the shared-memory tile
//     kernel and tlist holds their indices (ndense of them); slist holds the
//     B positions of the other cells (nsparse of them).
//   * per-replicate grid descriptors.
//
// Record positions: every hi part is an integer multiple of q with magnitude
// below 2^23 q, so hi_i - hi_j is exact in FP32 for any two cells of a
// replicate, and a pair's relative vector (hi_i - hi_j) + (lo_i - lo_j) is
// exact up to its final rounding.  Candidate tests use the hi parts with a
// margin of 2q.
#pragma once

#include <cmath>
#include <cstdint>
#include <string>

#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace mk {

enum Mode { kFP64 = 0, kMixedFP64Pos = 1, kMixedKahan = 2 };

constexpr int kScanThreads = 512;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;  // voxels per scan block

// Dense-tile force kernels: one warp per voxel of a dense tile (any tile), or
// one block per interior tile with its halo staged in shared memory.
constexpr int kMaxTypes = 16;  // cell types carried in 4 bits of the force record

constexpr int kTileKernelVox = 0;
constexpr int kTileKernelCTA = 1;

// Device error flag bits (the host reports any of them as MECH_E_DEVICE_FLAG).
constexpr uint32_t kErrNonFinite = 1u;
constexpr uint32_t kErrIndex = 2u;
constexpr uint32_t kErrTimeout = 4u;



struct GridDev {
    double lo[3];
    double h, inv_h;   // voxel side and its FP64 reciprocal (1/h rounded once)
    float lo_f[3];     // (float)lo
    float h_f, inv_h_f;  // (float)h, (float)(1/h)
    int32_t n[3];
    uint32_t vbase;    // first global voxel index of this replicate
    uint32_t cbase;    // first cell (same in caller and voxel order)
    uint32_t ncell;
    int32_t nt[3];     // tiles per axis
    uint32_t tbase;    // first global tile index of this replicate
    double whi[3];     // high corner of the domain box (the low corner is lo): the wall planes
    float whi_f[3];    // (float)whi
    double oc[3];      // grid centre: origin of the record positions
    float oc_hi[3], oc_lo[3];  // the centre as an exact FP32 pair
    float q, inv_q;    // grid of the hi parts (a power of two)
    float qs;          // q / 2^15: unit of the 16-bit position residuals
    float qm;          // candidate-test margin (>= 2 q)
    // The centre in fixed point, units of q / 2^24 (oc_fix = round(oc 2^24 / q)),
    // for an FP64 position's split into hi + lo with integer arithmetic;
    // fix_ok = 0 where a coordinate's fixed-point value could reach 2^61.
    long long oc_fix[3];
    int32_t qexp;      // q = 2^qexp
    int32_t fix_ok;
    float qf24;        // q / 2^24
};

// Position relative to the grid centre -> hi on the q grid (|hi| < 2^23 q);
// the residual r - hi is at most q/2.  A cell beyond 2^23 q (far outside its
// grid) keeps hi = r and lo = 0: its pair vectors are rounded once.
__device__ __forceinline__ float quantize_hi(float r, float q, float inv_q) {
    const float t = r * inv_q;
    return fabsf(t) < 8388608.f ? rintf(t) * q : r;
}

// FP64 position x -> hi + lo relative to the grid centre, without FP64
// arithmetic (this GPU's FP64 pipe runs at 1/64 of the FP32 rate): x is
// rounded to a multiple of q / 2^24 as a 64-bit integer X (from its exponent
// and mantissa), D = X - oc_fix, hi = round(D / 2^24) q (exact, |hi| < 2^23 q)
// and lo = (D - 2^24 round(D / 2^24)) q / 2^24 (exact: |lo| <= q / 2).  The
// error against x - oc is at most q / 2^24, far below the 16-bit residual
// stored in the record (q / 2^15).  Returns false (the caller then takes the
// FP64 route) for a non-finite x, |X| >= 2^62, or |hi| >= 2^23 q.
__device__ __forceinline__ bool split_fixed(double x, const GridDev& g, int d, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FFull);
    if (E == 0x7FF) return false;
    long long X = 0;
    if (E != 0) {  // (a subnormal x counts as 0)
        const long long M = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);  // 53 bits
        const int sh = E - 1075 - g.qexp + 24;  // x / (q 2^-24) = M 2^sh
        if (sh > 8) return false;
        if (sh >= 0) X = M << sh;
        else if (sh > -63) X = (M + (1ll << (-sh - 1))) >> (-sh);  // to nearest, ties up
        if (b >> 63) X = -X;
    }
    const long long D = X - g.oc_fix[d];
    const long long H = (D + (1ll << 23)) >> 24;  // nearest multiple of 2^24 (ties up)
    if (H >= (1ll << 23) || H <= -(1ll << 23)) return false;
    const int L = (int)(D - H * (1ll << 24));  // in [-2^23, 2^23)
    hi = (float)(int)H * g.q;
    lo = (float)L * g.qf24;
    return true;
}

// FP64 <-> compensated FP32 pair without FP64 arithmetic (this GPU's FP64
// pipe runs at 1/64 of the FP32 rate; these run where positions cross the
// host boundary).  Both give bit for bit the IEEE results of the FP64 forms
// they replace, and return false (the caller then takes the FP64 form) where
// that would need more care: zero, subnormal or non-finite operands, a float
// overflow, or a scale outside the normal range.
//
// x -> (xh, c) with xh = RN_f32(x) and c = RN_f32(xh - x): the 53-bit
// significand S of x is rounded to 24 bits (ties to even); r = S24 2^29 - S
// is then xh - x in units of 2^(E - 1075), a 30-bit integer, and c is its
// float conversion (one rounding) times that power of two (exact).
__device__ __forceinline__ bool split_double_f32(double x, float& xh, float& c) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7FFull);
    if (E < 949 || E == 0x7FF) return false;  // |x| < 2^-74, or not finite
    const long long S = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
    long long S24 = S >> 29;
    const long long R = S & 0x1FFFFFFFll;
    if (R > 0x10000000ll || (R == 0x10000000ll && (S24 & 1))) ++S24;
    const int r = (int)((S24 << 29) - S);  // |r| <= 2^28
    int ef = E - 1023;
    long long S24m = S24;
    if (S24 == (1ll << 24)) {
        S24m = 1ll << 23;
        ++ef;
    }
    if (ef > 127) return false;
    const unsigned int sgn = (unsigned int)(b >> 63) << 31;
    xh = __uint_as_float(sgn | ((unsigned int)(ef + 127) << 23) | (unsigned int)(S24m - (1ll << 23)));
    if (r == 0) {
        c = 0.0f;
    } else {
        const float scale = __uint_as_float((unsigned int)(E - 1075 + 127) << 23);  // 2^(E - 1075)
        c = __uint_as_float(__float_as_uint(__int2float_rn(r) * scale) ^ sgn);
    }
    return true;
}

// (xh, c) -> (double)xh - (double)c, rounded to nearest (ties to even): both
// are 24-bit significands S1 2^k1, S2 2^k2; for 0 <= k1 - k2 <= 39 the exact
// difference is a 64-bit integer times 2^k2, normalised and rounded here.
__device__ __forceinline__ bool join_f32_double(float xh, float c, double& x) {
    const unsigned int b1 = __float_as_uint(xh), b2 = __float_as_uint(c);
    const int E1 = (int)((b1 >> 23) & 0xFFu);
    if (E1 == 0 || E1 == 0xFF) return false;
    const long long S1 = (long long)((b1 & 0x7FFFFFu) | 0x800000u);
    const unsigned long long s1 = (unsigned long long)(b1 >> 31);
    if ((b2 & 0x7FFFFFFFu) == 0u) {  // c = 0: x = xh exactly
        x = __longlong_as_double(
            (long long)((s1 << 63) | ((unsigned long long)(E1 + 896) << 52) | ((unsigned long long)(S1 - (1ll << 23)) << 29)));
        return true;
    }
    const int E2 = (int)((b2 >> 23) & 0xFFu);
    if (E2 == 0 || E2 == 0xFF) return false;
    const int g = E1 - E2;
    if (g < 0 || g > 39) return false;
    const long long S2 = (long long)((b2 & 0x7FFFFFu) | 0x800000u);
    const long long X = ((b1 >> 31) ? -S1 : S1) * (1ll << g) - ((b2 >> 31) ? -S2 : S2);
    if (X == 0) {
        x = 0.0;
        return true;
    }
    const unsigned long long sg = X < 0 ? 1ull : 0ull;
    unsigned long long U = (unsigned long long)(X < 0 ? -X : X);
    const int lz = __clzll((long long)U);
    U <<= lz;
    const unsigned long long rnd = U & 0x7FFull;
    unsigned long long mant = (U >> 11) & 0xFFFFFFFFFFFFFull;
    long long ex = 1023 + 63 - lz + (E2 - 150);
    if (rnd > 0x400ull || (rnd == 0x400ull && (mant & 1ull))) {
        if (++mant == (1ull << 52)) {
            mant = 0;
            ++ex;
        }
    }
    if (ex <= 0 || ex >= 0x7FF) return false;
    x = __longlong_as_double((long long)((sg << 63) | ((unsigned long long)ex << 52) | mant));
    return true;
}

// 16-bit fixed point with offset 2^15: v in [-1, 1) units -> [0, 65535].
__device__ __forceinline__ uint32_t fix16(float v_units) {
    const float t = fminf(fmaxf(rintf(v_units * 32768.f), -32768.f), 32767.f);
    return (uint32_t)((int)t + 32768);
}

// 16-bit field u (offset 2^15) scaled by s (a power of two), exactly:
// 0x4B000000 | u is the float 2^23 + u, and (2^23 + u) s - (2^23 + 2^15) s is
// (u - 2^15) s without rounding.
__device__ __forceinline__ float unfix16(uint32_t u16, float s) {
    return fmaf(__int_as_float(0x4B000000u | u16), s, -8421376.f * s);
}

// 12-bit field u (offset 2^11) scaled by s (a power of two), exactly (as
// unfix16: (2^23 + u) s - (2^23 + 2^11) s).
__device__ __forceinline__ float unfix12(uint32_t u12, float s) {
    return fmaf(__int_as_float(0x4B000000u | u12), s, -8390656.f * s);
}

// Scale of the radius residual: ulp(R) / 2^11 for a normal R > 2^-91.
__device__ __forceinline__ float rlo_scale(float R) {
    return __int_as_float((int)(__float_as_uint(R) & 0x7F800000u) - ((23 + 11) << 23));
}

// Position residuals and radius residual of a record: {x_lo, y_lo, z_lo, R_lo}
// (qs = q / 2^15).
__device__ __forceinline__ float4 record_lo(const float4 p, const float4 c, float qs) {
    const uint32_t wxy = __float_as_uint(c.z), wzr = __float_as_uint(c.w);
    return make_float4(unfix16(wxy & 0xFFFFu, qs), unfix16(wxy >> 16, qs), unfix16(wzr & 0xFFFFu, qs),
                       unfix12((wzr >> 16) & 0xFFFu, rlo_scale(p.w)));
}

// Cell type carried in a record's second half (0..15).
__device__ __forceinline__ uint32_t record_type(const float4 c) { return __float_as_uint(c.w) >> 28; }

// Upper 16 bits of lo_zr for a radius R (FP64) and a type: the residual
// R - (float)R in units of ulp(R) / 2^11, offset 2^11, and the type above it.
__host__ __device__ inline uint32_t radius_type_bits(double R, float Rf, uint32_t type) {
    int e2 = 0;
    frexpf(Rf, &e2);  // Rf = f 2^e2, f in [0.5, 1): ulp(Rf) = 2^(e2 - 24)
    const double units = (R - (double)Rf) / ldexp(1.0, e2 - 24);
    double t = units * 2048.0;
    t = t < -2048.0 ? -2048.0 : (t > 2047.0 ? 2047.0 : t);
    const long long L = llround(t);
    return ((uint32_t)(L + 2048) | (type << 12)) << 16;
}

// Error-free sum: s + e == a + b exactly (Knuth).
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

struct StateBuf {
    double* pos64;
    float* posf;
    float* comp;
    double* vp64;
    float* vpf;
    uint32_t* id;
    float4* rec;       // force records, two float4 per cell (see the layout above)
};

struct StepArgs {
    int mode;
    uint32_t n;
    uint32_t npad;
    int nrep;
    const GridDev* grids;
    StateBuf A, B;
    uint32_t* key;
    uint32_t* vkey_s;
    uint32_t* perm;
    unsigned long long* tmp;
    uint32_t* count_cur;
    uint32_t* count_nxt;
    uint32_t* bcount_cur;  // cells per scan block (kScanTile voxels), this step and the next
    uint32_t* bcount_nxt;
    uint32_t* start;
    uint32_t* occ;         // 1 bit per voxel: count > 0 (written by the scan)
    const double* R64;    // FP64 parameters in caller order (FP64 mode)
    const double* ccr64;
    const double* cca64;
    float A_f, dt_f;
    float A2m1_f;          // A^2 - 1 (rounded once)
    double A_d, dt_d;
    int integrate;         // 1: AB2 update; 0: velocities only (positions kept)
    // velocity variants (off: ntypes 0, walls 0)
    int ntypes;            // > 0: per-type adhesion affinity, tables of 16 x 16 entries
    const float* aff_f;    // affinity a[t_i][t_j] at 16 t_i + t_j (FP32 modes)
    const double* aff_d;   // the same in FP64 (FP64 mode)
    int walls;             // enabled faces: bit f for -x, +x, -y, +y, -z, +z
    double c_wall;         // wall coefficient (um/min)
    float* vout_f;         // velocities-only output, B order (mixed modes)
    double* vout_d;        // velocities-only output, B order (FP64 mode)
    uint32_t* err;
    // tiles
    int ltx, lty, ltz;     // log2 of the tile dimensions (voxels)
    int use_tiles;         // 1: dense tiles go to a dense-tile kernel
    int tile_kernel;       // kTileKernelVox (warp per voxel) or kTileKernelCTA (block per interior tile)
    uint32_t ntiles;       // tiles over all replicates
    uint32_t dense_min;    // a tile with at least this many cells is dense
    uint32_t* tcount_cur;
    uint32_t* tcount_nxt;
    uint8_t* tdense;
    uint32_t* tlist;
    uint32_t* ndense;
    uint2* slist;          // {B position | alone << 31, voxel key} of the cells outside dense tiles
                           // (alone: no other cell in its voxel)
    uint32_t* nsparse;     // [0] sparse-list length, [1] tile cursor of the tile kernel
                           // (both zeroed by k_tile_classify)
    float cut_eps;         // candidate-test margin for FP32 rounding (added to each grid's qm)
    unsigned long long wait_ns;  // time limit of every device-side wait
    uint32_t fault;        // host-armed fault injection (kFault* bits)
};

// Host-armed fault injection (never set in normal runs).
constexpr uint32_t kFaultTileWait = 1u;  // the tile kernel's TMA barrier expects 16 bytes too many

// Streaming multiprocessors of the current device (queried once per device;
// grid caps of the grid-stride kernels are multiples of it).
int device_sms();

// ---- launch wrappers (mech_bin.cu) ----
cudaError_t launch_zero_u32(uint32_t* p, size_t count, cudaStream_t s);
// Keys and histograms of the cells in A order, and the histogram's scan-block
// sums (bcount_cur) for the step's scan.
cudaError_t launch_keys(const StepArgs& a, int grid, uint32_t vpad, cudaStream_t s);
cudaError_t launch_scan(const uint32_t* count, uint32_t vpad, uint32_t* bsum, uint32_t* start,
                        uint32_t* zero_word, uint32_t* occ, cudaStream_t s);
// The same scan when bsum already holds the cells of each block of kScanTile
// voxels (counted with the histogram): no reduce pass; zero_blocks (the next
// step's block sums) is cleared on the way.
cudaError_t launch_scan_blocks(const uint32_t* count, uint32_t vpad, uint32_t* bsum, uint32_t* zero_blocks,
                               uint32_t* start, uint32_t* zero_word, uint32_t* occ, cudaStream_t s);
cudaError_t launch_scatter(const StepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_canon(const StepArgs& a, int grid, cudaStream_t s);
// Positions in caller order (3n doubles into out); stage: 3n doubles of
// device scratch; scratch: scratch_cap bytes (256-aligned) of device scratch,
// at least unpermute_scratch_bytes(n), about 2n (cudaErrorInvalidValue
// otherwise).
size_t unpermute_scratch_bytes(uint32_t n);
cudaError_t launch_unpermute_pos(const StepArgs& a, const StateBuf& st, double* out, double* stage, void* scratch,
                                 size_t scratch_cap, cudaStream_t s);

// ---- dynamic population, between steps (mech_api.cu: mech_remove_cells /
// mech_add_cells) ----
// flags[i] = (alive[i] != 0) for i < n, 0 for n <= i < pad (a scan input).
cudaError_t launch_alive_flags(const uint8_t* alive, uint32_t n, uint32_t pad, uint32_t* flags, cudaStream_t s);
// flags[q] = (alive[st.id[q]] != 0) in state order, 0 up to pad.
cudaError_t launch_keep_flags(const StepArgs& a, const StateBuf& st, const uint8_t* alive, uint32_t pad,
                              uint32_t* flags, cudaStream_t s);
// Survivors of a.A end in slots [0, n2) in place: the survivors at or above
// n2 fill the dead slots below n2 (keep_pref: exclusive prefix of the keep
// flags over the state order; hole: scratch of n2 entries), then every
// survivor takes caller index newid[id] (exclusive prefix of the alive flags
// over the caller order).  Every state array is moved, whatever the mode.
cudaError_t launch_remove_in_place(const StepArgs& a, const uint8_t* alive, const uint32_t* keep_pref,
                                   const uint32_t* newid, uint32_t n2, uint32_t* hole, cudaStream_t s);
// FP64 parameters of the survivors (caller order) into io[0..np), io[np..2np),
// io[2np..3np) at their new caller index.
cudaError_t launch_compact_params(const StepArgs& a, const uint8_t* alive, const uint32_t* newid, double* io,
                                  cudaStream_t s);
// New cell k of m goes to slot and caller index dst[k] of st: FP64
// parameters (into R64, ccr64, cca64, caller order), force record (with its
// type types[k], or 0 if types is null), position
// (rounded as by mech_write_positions) and zero previous velocity, from io
// (positions at [0, 3m), R, ccr, cca at [3m, 4m), [4m, 5m), [5m, 6m)).
cudaError_t launch_append_state(const StepArgs& a, const StateBuf& st, const double* io, const uint32_t* dst,
                                const uint32_t* types, uint32_t m, double* R64, double* ccr64, double* cca64,
                                cudaStream_t s);
// Batches: order-preserving removal from a.A into a.B (dst: exclusive prefix
// of the keep flags over the state order), every replicate staying one range.
cudaError_t launch_compact_state(const StepArgs& a, const uint8_t* alive, const uint32_t* dst, const uint32_t* newid,
                                 cudaStream_t s);
// Batches: every cell of replicate r moves up by shift[r], state A -> B and
// its FP64 parameters into io[0..np), io[np..2np), io[2np..3np).
cudaError_t launch_shift(const StepArgs& a, const uint32_t* shift, double* io, cudaStream_t s);
cudaError_t launch_unpermute_vel(const StepArgs& a, const StateBuf& st, const float* vf, const double* vd,
                                 double* out, cudaStream_t s);
cudaError_t launch_load_pos(const StepArgs& a, const StateBuf& st, const double* in, int raw_kahan,
                            const double* comp_in, cudaStream_t s);
cudaError_t launch_load_vprev(const StepArgs& a, const StateBuf& st, const double* in, cudaStream_t s);

// ---- error reporting of the C ABI (mech_api.cu): sets mech_last_error ----
int record_error(int code, const std::string& msg);

// ---- launch wrappers (mech_force.cu) ----
// Velocity + AB2 of every cell: FP64 kernel, or (mixed modes) the tile
// classification, the shared-memory tile kernel for dense tiles and the
// thread-per-cell kernel for the rest.  Each phase is a separate launch so
// that it can be timed; `ev` (may be null) receives an event between phases.
cudaError_t launch_tile_classify(const StepArgs& a, cudaStream_t s);
cudaError_t launch_force_tiles(const StepArgs& a, int grid, cudaStream_t s);
cudaError_t launch_sparse_list(const StepArgs& a, int grid, cudaStream_t s);
// Neighbour statistics of the voxel order in a.B (after a binning pass) from
// FP64 positions in caller order: out[0] += candidates, out[1] += ordered
// interacting pairs.
cudaError_t launch_pair_stats(const StepArgs& a, const double* xyz, unsigned long long* out, int grid,
                              cudaStream_t s);
cudaError_t launch_force_cells(const StepArgs& a, int grid, int block, cudaStream_t s);
int force_max_blocks_per_sm(int mode, int block);
int tile_kernel_grid(const StepArgs& a, int sms);
bool tile_shape_supported(int ltx, int lty, int ltz);

// ---- small device helpers shared by the kernel files ----
__device__ __forceinline__ int rep_of_cell(const GridDev* g, int nrep, uint32_t q) {
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g[mid].cbase <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Voxel index along one axis from an FP64 coordinate: floor((x - lo) * inv_h)
// with two IEEE roundings and no contraction, clamped into [0, n-1] (NaN -> 0).
__device__ __forceinline__ int axis_index_f64(double x, double lo, double inv_h, int n) {
    double t = __dmul_rn(__dsub_rn(x, lo), inv_h);
    double f = floor(t);
    if (!(f >= 0.0)) return 0;
    if (f >= (double)(n - 1)) return n - 1;
    return (int)f;
}

// Same decision taken in FP32 (positions held in FP32, or rounded to FP32).
__device__ __forceinline__ int axis_index_f32(float x, float lo, float inv_h, int n) {
    float t = __fmul_rn(__fsub_rn(x, lo), inv_h);
    float f = floorf(t);
    if (!(f >= 0.0f)) return 0;
    if (f >= (float)(n - 1)) return n - 1;
    return (int)f;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int rep_of_tile(const GridDev* g, int nrep, uint32_t t) {
    int lo = 0, hi = nrep - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (g[mid].tbase <= t) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint32_t tile_index(const GridDev& g, int ix, int iy, int iz, int ltx, int lty,
                                               int ltz) {
    return g.tbase + (uint32_t)(ix >> ltx) +
           (uint32_t)g.nt[0] * ((uint32_t)(iy >> lty) + (uint32_t)g.nt[1] * (uint32_t)(iz >> ltz));
}

// Voxel key of the cell at state index i (positions in state buffer st).
__device__ __forceinline__ uint32_t cell_key(int mode, const GridDev& g, const StateBuf& st, uint32_t npad,
                                             uint32_t i, int& ix, int& iy, int& iz) {
    if (mode == kFP64) {
        ix = axis_index_f64(st.pos64[i], g.lo[0], g.inv_h, g.n[0]);
        iy = axis_index_f64(st.pos64[npad + i], g.lo[1], g.inv_h, g.n[1]);
        iz = axis_index_f64(st.pos64[2 * (size_t)npad + i], g.lo[2], g.inv_h, g.n[2]);
    } else if (mode == kMixedFP64Pos) {
        ix = axis_index_f32(__double2float_rn(st.pos64[i]), g.lo_f[0], g.inv_h_f, g.n[0]);
        iy = axis_index_f32(__double2float_rn(st.pos64[npad + i]), g.lo_f[1], g.inv_h_f, g.n[1]);
        iz = axis_index_f32(__double2float_rn(st.pos64[2 * (size_t)npad + i]), g.lo_f[2], g.inv_h_f, g.n[2]);
    } else {
        ix = axis_index_f32(st.posf[i], g.lo_f[0], g.inv_h_f, g.n[0]);
        iy = axis_index_f32(st.posf[npad + i], g.lo_f[1], g.inv_h_f, g.n[1]);
        iz = axis_index_f32(st.posf[2 * (size_t)npad + i], g.lo_f[2], g.inv_h_f, g.n[2]);
    }
    return g.vbase + (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy + (uint32_t)g.n[1] * (uint32_t)iz);
}

// Warp-aggregated histogram increment: lanes with equal keys share one atomic.
// All 32 lanes must call it; lanes with valid == false take no slot.
__device__ __forceinline__ uint32_t warp_count(uint32_t* count, uint32_t key, bool valid) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t k = valid ? key : 0xFFFFFFFFu;
    uint32_t grp = __match_any_sync(0xFFFFFFFFu, k);
    uint32_t leader = __ffs(grp) - 1;
    uint32_t base = 0;
    if (valid && lane == leader) base = atomicAdd(&count[key], (uint32_t)__popc(grp));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + (uint32_t)__popc(grp & lanemask_lt());
}

// Warp-aggregated increment without a slot (tile histogram).
__device__ __forceinline__ void warp_add(uint32_t* count, uint32_t key, bool valid) {
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t k = valid ? key : 0xFFFFFFFFu;
    uint32_t grp = __match_any_sync(0xFFFFFFFFu, k);
    if (valid && lane == (uint32_t)(__ffs(grp) - 1)) atomicAdd(&count[key], (uint32_t)__popc(grp));
}

// Affinity factor of a pair of types (1 when the affinity is off).
__device__ __forceinline__ float affinity_f(const StepArgs& a, uint32_t ti, uint32_t tj) {
    return a.ntypes > 0 ? __ldg(&a.aff_f[ti * kMaxTypes + tj]) : 1.0f;
}

// Domain-wall terms of one cell (velocity variant), added to acc in face
// order -x, +x, -y, +y, -z, +z, in FP64 with the definition's operations:
// d_w = inward distance of the centre x from the face; if d_w < R,
// t = 1 - d_w / R (t = 1 for d_w <= 0) and acc += c_w t^2 along the inward
// normal.
__device__ __forceinline__ void wall_terms(const StepArgs& a, const GridDev& g, const double x[3], double R,
                                           double acc[3]) {
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (!(a.walls & (1 << f))) continue;
        const int axis = f >> 1;
        const bool high = (f & 1) != 0;
        const double dw = high ? __dsub_rn(g.whi[axis], x[axis]) : __dsub_rn(x[axis], g.lo[axis]);
        if (!(dw < R)) continue;
        const double t = dw > 0.0 ? __dsub_rn(1.0, __ddiv_rn(dw, R)) : 1.0;
        const double push = __dmul_rn(a.c_wall, __dmul_rn(t, t));
        acc[axis] = high ? __dsub_rn(acc[axis], push) : __dadd_rn(acc[axis], push);
    }
}

// Whether an FP32 position may lie within R + 1 um of an enabled face (a
// conservative test: the FP32 rounding of a coordinate is far below 1 um).
__device__ __forceinline__ bool near_wall(const StepArgs& a, const GridDev& g, const float xf[3], float R) {
    bool near = false;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
        if (!(a.walls & (1 << f))) continue;
        const int axis = f >> 1;
        const float dw = (f & 1) ? g.whi_f[axis] - xf[axis] : xf[axis] - g.lo_f[axis];
        near = near || dw < R + 1.0f;
    }
    return near;
}

}  // namespace mk
