// Neighbour-gather velocity and AB2 integration (steps 2 and 3 of the
// mechanics update; the paper's "update velocity" region, Sec. 5.4).
//
// Work split: one thread per cell, threads in voxel order.  Each voxel thus
// gets exactly as many threads as it holds cells (empty voxels get none, the
// GPU form of the paper's non-empty-voxel list), consecutive threads share
// neighbour voxels (the locality the paper's voxel-ordered loop was after),
// and a dense core is spread over as many warps as it has cells / 32.
//
// For cell i in voxel (ix, iy, iz) the 27 neighbour voxels are visited in
// lexicographic (dz, dy, dx) order; the three voxels of one (dy, dz) row are
// contiguous in the sorted arrays.  Candidate positions are FP32 offsets from
// their own voxel origin, so the pair vector is (p_i - off) - p_j with
// off = (dx, dy, dz) h: no FP64 arithmetic in the candidate loop.
#include "mech_internal.cuh"

namespace mk {

namespace {

constexpr int kForceBlock = 256;

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

// ---------------------------------------------------------------- FP32 ----
// Mixed modes: pair arithmetic and the sum in FP32; positions in FP64
// (MODE = kMixedFP64Pos) or FP32 + Kahan compensation (MODE = kMixedKahan).
template <int MODE>
__global__ void __launch_bounds__(kForceBlock) k_force_mixed(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const float A = a.A_f;
    for (uint32_t base = warp * 32u; base < a.n; base += nwarps * 32u) {
        const uint32_t q = base + lane;
        const bool valid = q < a.n;
        uint32_t nkey = 0;
        if (valid) {
            const int r = rep_of_cell(a.grids, a.nrep, q);
            const GridDev& g = a.grids[r];
            const Cell3 c = decode(a.vkey_s[q], g);
            const float4 pi = a.B.cand[q];
            const float2 ci = a.B.candp[q];
            const float h = g.h_f;
            float ax = 0.f, ay = 0.f, az = 0.f;
            for (int dz = -1; dz <= 1; ++dz) {
                const int jz = c.iz + dz;
                if (jz < 0 || jz >= g.n[2]) continue;
                const float oz = pi.z - (float)dz * h;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int jy = c.iy + dy;
                    if (jy < 0 || jy >= g.n[1]) continue;
                    const float oy = pi.y - (float)dy * h;
                    const uint32_t row = g.vbase + (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
                    const int jx0 = c.ix > 0 ? c.ix - 1 : 0;
                    const int jx1 = c.ix + 1 < g.n[0] ? c.ix + 1 : g.n[0] - 1;
                    uint32_t s = a.start[row + jx0];
                    for (int jx = jx0; jx <= jx1; ++jx) {
                        const uint32_t e = a.start[row + jx + 1];
                        const float ox = pi.x - (float)(jx - c.ix) * h;
                        for (uint32_t j = s; j < e; ++j) {
                            const float4 pj = a.B.cand[j];
                            const float rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
                            const float d2 = rx * rx + ry * ry + rz * rz;
                            const float S = pi.w + pj.w;
                            const float AS = A * S;
                            if (d2 < AS * AS && d2 > 0.f) {
                                const float2 cj = a.B.candp[j];
                                const float rd = rsqrtf(d2);
                                const float d = d2 * rd;
                                const float ta = 1.f - __fdividef(d, AS);
                                float cf = -(ci.y * cj.y) * (ta * ta);
                                if (d < S) {
                                    const float t = 1.f - __fdividef(d, S);
                                    cf += (ci.x * cj.x) * (t * t);
                                }
                                const float sc = cf * rd;
                                ax += sc * rx;
                                ay += sc * ry;
                                az += sc * rz;
                            }
                        }
                        s = e;
                    }
                }
            }
            // ---- AB2 epilogue: read the A-order state of this cell, write B ----
            const uint32_t src = a.perm[q];
            const size_t np = a.npad;
            const float v[3] = {ax, ay, az};
            bool finite = true;
            float xf[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float vp = a.A.vpf[d * np + src];
                const float inc = a.dt_f * (1.5f * v[d] - 0.5f * vp);
                if (MODE == kMixedFP64Pos) {
                    const double x = a.A.pos64[d * np + src];
                    const double xn = a.integrate ? __dadd_rn(x, (double)inc) : x;
                    a.B.pos64[d * np + q] = xn;
                    xf[d] = __double2float_rn(xn);
                    finite = finite && isfinite(xn);
                } else {
                    float xh = a.A.posf[d * np + src];
                    float cc = a.A.comp[d * np + src];
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
                a.B.vpf[d * np + q] = a.integrate ? v[d] : vp;
                if (!a.integrate) a.vout_f[d * np + q] = v[d];
                finite = finite && isfinite(v[d]);
            }
            a.B.id[q] = a.A.id[src];
            if (!finite) atomicOr(a.err, kErrNonFinite);
            const int ix = axis_index_f32(xf[0], g.lo_f[0], g.inv_h_f, g.n[0]);
            const int iy = axis_index_f32(xf[1], g.lo_f[1], g.inv_h_f, g.n[1]);
            const int iz = axis_index_f32(xf[2], g.lo_f[2], g.inv_h_f, g.n[2]);
            nkey = g.vbase + (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy + (uint32_t)g.n[1] * (uint32_t)iz);
        }
        // histogram of the next step's binning, fused here
        const uint32_t slot = warp_count(a.count_nxt, nkey, valid);
        if (valid) {
            a.key[q] = nkey;
            a.slot[q] = slot;
        }
    }
}

// ---------------------------------------------------------------- FP64 ----
// All-FP64 mode.  An FP32 test with a relative margin of 1e-4 on the squared
// cutoff discards candidates that are certainly out of range; the survivors
// are evaluated in FP64 from the FP64 positions and parameters with the same
// operations, in the same order, as the definition (no contraction, IEEE sqrt
// and division), and summed in the definition's candidate order.
__global__ void __launch_bounds__(kForceBlock) k_force_fp64(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const float A = a.A_f;
    const double Ad = a.A_d;
    const size_t np = a.npad;
    for (uint32_t base = warp * 32u; base < a.n; base += nwarps * 32u) {
        const uint32_t q = base + lane;
        const bool valid = q < a.n;
        uint32_t nkey = 0;
        if (valid) {
            const int r = rep_of_cell(a.grids, a.nrep, q);
            const GridDev& g = a.grids[r];
            const Cell3 c = decode(a.vkey_s[q], g);
            const float4 pi = a.B.cand[q];
            const uint32_t src = a.perm[q];
            const uint32_t idi = a.A.id[src];
            const double xi = a.A.pos64[src], yi = a.A.pos64[np + src], zi = a.A.pos64[2 * np + src];
            const double Ri = a.R64[idi], ccri = a.ccr64[idi], ccai = a.cca64[idi];
            const float h = g.h_f;
            double ax = 0.0, ay = 0.0, az = 0.0;
            for (int dz = -1; dz <= 1; ++dz) {
                const int jz = c.iz + dz;
                if (jz < 0 || jz >= g.n[2]) continue;
                const float oz = pi.z - (float)dz * h;
                for (int dy = -1; dy <= 1; ++dy) {
                    const int jy = c.iy + dy;
                    if (jy < 0 || jy >= g.n[1]) continue;
                    const float oy = pi.y - (float)dy * h;
                    const uint32_t row = g.vbase + (uint32_t)g.n[0] * ((uint32_t)jy + (uint32_t)g.n[1] * (uint32_t)jz);
                    const int jx0 = c.ix > 0 ? c.ix - 1 : 0;
                    const int jx1 = c.ix + 1 < g.n[0] ? c.ix + 1 : g.n[0] - 1;
                    uint32_t s = a.start[row + jx0];
                    for (int jx = jx0; jx <= jx1; ++jx) {
                        const uint32_t e = a.start[row + jx + 1];
                        const float ox = pi.x - (float)(jx - c.ix) * h;
                        for (uint32_t j = s; j < e; ++j) {
                            if (j == q) continue;
                            const float4 pj = a.B.cand[j];
                            const float rx = ox - pj.x, ry = oy - pj.y, rz = oz - pj.z;
                            const float d2f = rx * rx + ry * ry + rz * rz;
                            const float ASf = A * (pi.w + pj.w);
                            if (!(d2f <= ASf * ASf * 1.0001f + 1e-2f)) continue;
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
                            cf = __dsub_rn(cf, __dmul_rn(__dsqrt_rn(__dmul_rn(ccai, a.cca64[idj])), __dmul_rn(ta, ta)));
                            const double sc = __ddiv_rn(cf, d);
                            ax = __dadd_rn(ax, __dmul_rn(sc, dx));
                            ay = __dadd_rn(ay, __dmul_rn(sc, dy2));
                            az = __dadd_rn(az, __dmul_rn(sc, dz2));
                        }
                        s = e;
                    }
                }
            }
            const double v[3] = {ax, ay, az};
            const double xo[3] = {xi, yi, zi};
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
            a.B.id[q] = idi;
            if (!finite) atomicOr(a.err, kErrNonFinite);
            const int ix = axis_index_f64(xn[0], g.lo[0], g.inv_h, g.n[0]);
            const int iy = axis_index_f64(xn[1], g.lo[1], g.inv_h, g.n[1]);
            const int iz = axis_index_f64(xn[2], g.lo[2], g.inv_h, g.n[2]);
            nkey = g.vbase + (uint32_t)ix + (uint32_t)g.n[0] * ((uint32_t)iy + (uint32_t)g.n[1] * (uint32_t)iz);
        }
        const uint32_t slot = warp_count(a.count_nxt, nkey, valid);
        if (valid) {
            a.key[q] = nkey;
            a.slot[q] = slot;
        }
    }
}

}  // namespace

int force_max_blocks_per_sm(int mode, int block) {
    int nb = 0;
    if (mode == kFP64)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_fp64, block, 0);
    else if (mode == kMixedFP64Pos)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_mixed<kMixedFP64Pos>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_force_mixed<kMixedKahan>, block, 0);
    return nb > 0 ? nb : 1;
}

cudaError_t launch_force(const StepArgs& a, int grid, int block, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (a.mode == kFP64)
        k_force_fp64<<<grid, block, 0, s>>>(a);
    else if (a.mode == kMixedFP64Pos)
        k_force_mixed<kMixedFP64Pos><<<grid, block, 0, s>>>(a);
    else
        k_force_mixed<kMixedKahan><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace mk
