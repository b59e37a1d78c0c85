// Binning kernels of the mechanics step: voxel keys + histogram, exclusive
// scan, stable scatter into voxel order, and the host-order <-> voxel-order
// copies used by the read/write calls.
//
// The counting sort is the GPU form of the paper's locality lesson (Sec. 5.4):
// cells are re-stored every step in the order of the 3-D voxel mesh so that
// spatial neighbours are memory neighbours, and a voxel costs work only in
// proportion to the cells it holds.  Order inside a voxel is ascending caller
// index, which makes the permutation a function of the positions alone.
#include <algorithm>
#include <atomic>

#include "mech_internal.cuh"

namespace mk {

namespace {

__global__ void k_zero_u32(uint32_t* __restrict__ p, size_t count) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (; i < count; i += stride) p[i] = 0u;
}

// Step 1a (first step after a state change): key of every cell in A order and
// the histograms of voxels and tiles.  Loop is warp-uniform so that the
// aggregated atomics always run on full warps.
__global__ void k_keys(const StepArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t base = warp * 32u; base < a.n; base += nwarps * 32u) {
        const uint32_t i = base + lane;
        const bool valid = i < a.n;
        uint32_t key = 0, tile = 0;
        if (valid) {
            const int r = rep_of_cell(a.grids, a.nrep, i);
            const GridDev& g = a.grids[r];
            int ix, iy, iz;
            key = cell_key(a.mode, g, a.A, a.npad, i, ix, iy, iz);
            tile = tile_index(g, ix, iy, iz, a.ltx, a.lty, a.ltz);
        }
        warp_add(a.count_cur, key, valid);
        warp_add(a.tcount_cur, tile, valid);
        if (valid) a.key[i] = key;
    }
}

// ---- exclusive scan of the histogram (reduce, scan of block sums, down-sweep) ----

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* sh_warp, uint32_t* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh_warp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < nw ? sh_warp[lane] : 0u;
        uint32_t ws = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xFFFFFFFFu, ws, o);
            if (lane >= o) ws += y;
        }
        if (lane < nw) sh_warp[lane] = ws - w;
        if (lane == nw - 1) sh_warp[32] = ws;
    }
    __syncthreads();
    uint32_t r = sh_warp[wid] + x - v;
    *total = sh_warp[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ count,
                                                              uint32_t* __restrict__ bsum) {
    __shared__ uint32_t sh[33];
    const size_t base = (size_t)blockIdx.x * kScanTile;
    const uint4* c4 = reinterpret_cast<const uint4*>(count + base);
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
        uint4 q = c4[k * kScanThreads + threadIdx.x];
        s += q.x + q.y + q.z + q.w;
    }
    uint32_t tot;
    block_exclusive_scan(s, sh, &tot);
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

// One block scans the block sums in place (exclusive); it also clears one
// counter word for a later kernel of the same step (may be null).
__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* __restrict__ bsum, uint32_t nb,
                                                   uint32_t* __restrict__ zero_word) {
    __shared__ uint32_t sh[33];
    if (zero_word && threadIdx.x == 0) *zero_word = 0u;
    uint32_t carry = 0;
    for (uint32_t base = 0; base < nb; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint32_t v = i < nb ? bsum[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
}

// start[v] = sum_{u<v} count[u]; each thread owns 16 consecutive voxels, and
// writes their occupancy bits.  zero_blocks (may be null): the block's entry
// of another block-sum array is cleared.
__global__ void __launch_bounds__(kScanThreads) k_scan_down(const uint32_t* __restrict__ count,
                                                            const uint32_t* __restrict__ boff,
                                                            uint32_t* __restrict__ start,
                                                            uint16_t* __restrict__ occ16,
                                                            uint32_t* __restrict__ zero_blocks) {
    __shared__ uint32_t sh[33];
    if (zero_blocks && threadIdx.x == 0) zero_blocks[blockIdx.x] = 0u;
    const size_t base = (size_t)blockIdx.x * kScanTile + (size_t)threadIdx.x * kScanItems;
    const uint4* c4 = reinterpret_cast<const uint4*>(count + base);
    uint4 q[kScanItems / 4];
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
        q[k] = c4[k];
        s += q[k].x + q[k].y + q[k].z + q[k].w;
    }
    uint32_t tot;
    uint32_t run = boff[blockIdx.x] + block_exclusive_scan(s, sh, &tot);
    uint4* s4 = reinterpret_cast<uint4*>(start + base);
#pragma unroll
    for (int k = 0; k < kScanItems / 4; ++k) {
        uint4 o;
        o.x = run; run += q[k].x;
        o.y = run; run += q[k].y;
        o.z = run; run += q[k].z;
        o.w = run; run += q[k].w;
        s4[k] = o;
    }
    if (occ16) {  // occupancy bits of this thread's 16 voxels
        uint32_t m = 0;
#pragma unroll
        for (int k = 0; k < kScanItems / 4; ++k) {
            m |= (uint32_t)(q[k].x != 0) << (4 * k);
            m |= (uint32_t)(q[k].y != 0) << (4 * k + 1);
            m |= (uint32_t)(q[k].z != 0) << (4 * k + 2);
            m |= (uint32_t)(q[k].w != 0) << (4 * k + 3);
        }
        occ16[base / kScanItems] = (uint16_t)m;
    }
}

// Step 1c: every cell goes to start[key] + slot, carrying (id, A index).  The
// slot is taken by counting the voxel's histogram entry back down, which
// leaves the histogram zero for its reuse as the next step's accumulator; the
// slot order inside a voxel comes from the atomics and k_canon makes it
// canonical.
__global__ void __launch_bounds__(256) k_scatter(const StepArgs a) {
    // four cells per thread (256 apart) per round: their key loads, then their
    // atomics and start[] loads, are issued together
    constexpr uint32_t kPer = 4, kRound = 256u * kPer;
    for (uint32_t base = blockIdx.x * kRound; base < a.n; base += gridDim.x * kRound) {
        uint32_t k[kPer], id[kPer], left[kPer], st[kPer];
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            const uint32_t i = base + j * 256u + threadIdx.x;
            k[j] = i < a.n ? a.key[i] : 0u;
            id[j] = i < a.n ? a.A.id[i] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            const uint32_t i = base + j * 256u + threadIdx.x;
            left[j] = i < a.n ? atomicSub(&a.count_cur[k[j]], 1u) : 0u;  // cells of voxel k not yet placed
            st[j] = i < a.n ? a.start[k[j]] : 0u;
        }
#pragma unroll
        for (uint32_t j = 0; j < kPer; ++j) {
            const uint32_t i = base + j * 256u + threadIdx.x;
            if (i >= a.n) continue;
            const uint32_t dst = st[j] + left[j] - 1u;
            if (left[j] == 0u || dst >= a.n) {  // only after an earlier device error left the keys inconsistent
                atomicOr(a.err, kErrIndex);
                continue;
            }
            a.tmp[dst] = ((unsigned long long)id[j] << 32) | (unsigned long long)i;
        }
    }
}

// Step 1d: canonicalisation, one thread per scattered entry q.  The cell is
// ranked inside its voxel by caller index (ids are unique), which gives its
// final voxel-order position f; perm[f] (its A index), its key and its id are
// recorded, and its force record is gathered from its A position and written
// at f (position relative to the grid centre as hi on the q grid + 16-bit
// residual, radius, coefficient square roots).  The rest of the state
// (position, compensation, previous velocity) stays in A order: the force
// kernels read it at perm[f] for the AB2 update and write the new state at f.
// Cells that stay in their voxel keep their relative order, so both the reads
// at perm[f] and the writes at f are close to sequential.
__global__ void k_canon(const StepArgs a) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const unsigned long long e = a.tmp[q];
        const uint32_t id = (uint32_t)(e >> 32);
        const uint32_t src = (uint32_t)e;
        if (src >= a.n) {  // only after an earlier device error
            atomicOr(a.err, kErrIndex);
            continue;
        }
        // the cell's state at src is loaded before the ranking, whose loads it
        // does not depend on
        float xs[3] = {0.f, 0.f, 0.f}, cs[3] = {0.f, 0.f, 0.f};
        double xd[3] = {0.0, 0.0, 0.0};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (a.mode == kMixedKahan) {
                xs[d] = a.A.posf[d * np + src];
                cs[d] = a.A.comp[d * np + src];
            } else {
                xd[d] = a.A.pos64[d * np + src];
            }
        }
        const float4 pa = a.A.rec[2 * (size_t)src];
        const float4 qa = a.A.rec[2 * (size_t)src + 1];
        const uint32_t k = a.key[src];
        const uint32_t s = a.start[k], en = a.start[k + 1];
        uint32_t rank = 0;
        for (uint32_t t = s; t < en; ++t) rank += (uint32_t)((uint32_t)(a.tmp[t] >> 32) < id);
        const uint32_t f = s + rank;
        if (f >= a.n) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
        a.perm[f] = src;
        a.vkey_s[f] = k;
        a.B.id[f] = id;  // written here, so the next state's slot map is complete even if a force kernel aborts
        const int r = rep_of_cell(a.grids, a.nrep, f);
        const GridDev& g = a.grids[r];
        float hi[3], lo[3];
        if (a.mode == kMixedKahan) {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float xh = xs[d];
                const float c = cs[d];
                // value - centre = (x_hi - oc_hi) - (oc_lo + c), both sums error-free
                float e1, e2;
                const float s1 = two_sum(xh, -g.oc_hi[d], e1);
                const float sv = two_sum(s1, -__fadd_rn(g.oc_lo[d], c), e2);
                hi[d] = quantize_hi(sv, g.q, g.inv_q);
                lo[d] = __fadd_rn(__fsub_rn(sv, hi[d]), __fadd_rn(e1, e2));
            }
        } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double x = xd[d];
                if (g.fix_ok && split_fixed(x, g, d, hi[d], lo[d])) continue;
                const double rr = __dsub_rn(x, g.oc[d]);
                const double t = rint(__dmul_rn(rr, (double)g.inv_q));
                if (fabs(t) < 8388608.0) {
                    const double hd = __dmul_rn(t, (double)g.q);  // exact: integer times a power of two
                    hi[d] = (float)hd;
                    lo[d] = __double2float_rn(__dsub_rn(rr, hd));
                } else {
                    hi[d] = __double2float_rn(rr);
                    lo[d] = 0.f;
                }
            }
        }
        // radius, its residual and the coefficients travel with the record
        const uint32_t wxy = fix16(lo[0] * g.inv_q) | (fix16(lo[1] * g.inv_q) << 16);
        const uint32_t wzr = fix16(lo[2] * g.inv_q) | (__float_as_uint(qa.w) & 0xFFFF0000u);
        a.B.rec[2 * (size_t)f] = make_float4(hi[0], hi[1], hi[2], pa.w);
        a.B.rec[2 * (size_t)f + 1] = make_float4(qa.x, qa.y, __uint_as_float(wxy), __uint_as_float(wzr));
    }
}

// Voxel order -> caller order (positions), in two passes through buckets of
// 2,048 consecutive caller ids.  Pass 1, in slot order: each cell appends its
// position to its bucket's run of the staging buffer (a bucket holds exactly
// its 2,048 ids, so the runs need no counting pass; the order inside a run
// comes from atomics) and the id's low 11 bits beside it.  Pass 2, one block
// per bucket: the run is placed by those bits into shared memory and written
// out contiguously.  (A direct scatter through the ids, three 8-byte writes
// per cell at random places of the output, measured slower end to end.)
constexpr uint32_t kUpLog = 11, kUpIds = 1u << kUpLog;

__global__ void k_unpermute_pos_stage(const StepArgs a, const StateBuf st, uint32_t* __restrict__ cursor,
                                      double* __restrict__ stage, uint16_t* __restrict__ low) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = st.id[q];
        double x[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            if (a.mode == kMixedKahan) {
                const float xh = st.posf[(size_t)d * a.npad + q], c = st.comp[(size_t)d * a.npad + q];
                if (!join_f32_double(xh, c, x[d])) x[d] = __dsub_rn((double)xh, (double)c);
            } else {
                x[d] = st.pos64[(size_t)d * a.npad + q];
            }
        }
        if (id >= a.n) {  // only after an earlier device error
            atomicOr(a.err, kErrIndex);
            continue;
        }
        const uint32_t bkt = id >> kUpLog;
        const uint32_t k = atomicAdd(&cursor[bkt], 1u);
        const size_t r = ((size_t)bkt << kUpLog) + k;  // k < the bucket's id count (ids are a permutation)
        if (k >= kUpIds || r >= a.n) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) stage[3 * r + d] = x[d];
        low[r] = (uint16_t)(id & (kUpIds - 1u));
    }
}

__global__ void __launch_bounds__(256) k_unpermute_pos_place(uint32_t n, const double* __restrict__ stage,
                                                             const uint16_t* __restrict__ low,
                                                             double* __restrict__ out) {
    __shared__ double sh[3 * kUpIds];
    const size_t base = (size_t)blockIdx.x << kUpLog;
    const uint32_t cnt = (uint32_t)min((size_t)kUpIds, (size_t)n - base);
    for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) {
        const uint32_t j = low[base + k];
        if (j < cnt) {
#pragma unroll
            for (int d = 0; d < 3; ++d) sh[3 * j + d] = stage[3 * (base + k) + d];
        }
    }
    __syncthreads();
    for (uint32_t w = threadIdx.x; w < 3 * cnt; w += blockDim.x) out[3 * base + w] = sh[w];
}

__global__ void k_unpermute_vel(const StepArgs a, const StateBuf st, const float* __restrict__ vf,
                                const double* __restrict__ vd, double* __restrict__ out) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = st.id[q];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            out[3 * (size_t)id + d] = vd ? vd[(size_t)d * a.npad + q] : (double)vf[(size_t)d * a.npad + q];
    }
}

// Caller order -> current state order (positions).  raw_kahan: `in` holds the
// FP32 x_hi values and comp_in the compensations (exact state reload);
// otherwise `in` is a position value and the Kahan pair is built from it.
__global__ void k_load_pos(const StepArgs a, const StateBuf st, const double* __restrict__ in, int raw_kahan,
                           const double* __restrict__ comp_in) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = st.id[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = in[3 * (size_t)id + d];
            if (a.mode == kMixedKahan) {
                float xh, c;
                if (raw_kahan) {
                    xh = (float)x;
                    c = comp_in ? (float)comp_in[3 * (size_t)id + d] : 0.0f;
                } else if (!split_double_f32(x, xh, c)) {
                    xh = __double2float_rn(x);
                    c = __double2float_rn(__dsub_rn((double)xh, x));
                }
                st.posf[(size_t)d * a.npad + q] = xh;
                st.comp[(size_t)d * a.npad + q] = c;
            } else {
                st.pos64[(size_t)d * a.npad + q] = x;
            }
        }
    }
}

// ---- dynamic population ----
__global__ void k_alive_flags(const uint8_t* __restrict__ alive, uint32_t n, uint32_t pad, uint32_t* __restrict__ flags) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < pad; i += stride)
        flags[i] = (i < n && alive[i] != 0) ? 1u : 0u;
}

__global__ void k_keep_flags(const StepArgs a, const StateBuf st, const uint8_t* __restrict__ alive, uint32_t pad,
                             uint32_t* __restrict__ flags) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < pad; q += stride) {
        uint32_t f = 0u;
        if (q < a.n) {
            const uint32_t id = st.id[q];
            if (id < a.n) f = alive[id] != 0 ? 1u : 0u;
            else atomicOr(a.err, kErrIndex);  // only after an earlier device error
        }
        flags[q] = f;
    }
}

// Removal in place, in state order: the survivors end in slots [0, n2).  A
// dead slot q < n2 is a hole, numbered q - keep_pref[q] (dead slots before
// it); a surviving slot q >= n2 is a mover, numbered keep_pref[q] -
// keep_pref[n2]; mover k fills hole k.  Holes and movers are disjoint, so the
// moves need no second buffer, and only as many cells move as died below n2
// (the next binning restores the voxel order).
__global__ void k_list_holes(const StepArgs a, const uint8_t* __restrict__ alive, const uint32_t* __restrict__ keep_pref,
                             uint32_t n2, uint32_t* __restrict__ hole) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += stride) {
        const uint32_t id = a.A.id[q];
        if (id >= a.n) {  // only after an earlier device error
            atomicOr(a.err, kErrIndex);
            continue;
        }
        if (!alive[id]) hole[q - keep_pref[q]] = q;
    }
}

__global__ void k_fill_holes(const StepArgs a, const uint8_t* __restrict__ alive, const uint32_t* __restrict__ keep_pref,
                             uint32_t n2, const uint32_t* __restrict__ hole) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    const uint32_t base = keep_pref[n2];
    for (uint32_t q = n2 + blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = a.A.id[q];
        if (id >= a.n) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
        if (!alive[id]) continue;
        const uint32_t f = hole[keep_pref[q] - base];
        if (f >= n2) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a.A.pos64[d * np + f] = a.A.pos64[d * np + q];
            a.A.posf[d * np + f] = a.A.posf[d * np + q];
            a.A.comp[d * np + f] = a.A.comp[d * np + q];
            a.A.vp64[d * np + f] = a.A.vp64[d * np + q];
            a.A.vpf[d * np + f] = a.A.vpf[d * np + q];
        }
        a.A.rec[2 * (size_t)f] = a.A.rec[2 * (size_t)q];
        a.A.rec[2 * (size_t)f + 1] = a.A.rec[2 * (size_t)q + 1];
        a.A.id[f] = id;
    }
}

// Caller indices of the survivors in slots [0, n2): their rank among the
// survivors in caller order.
__global__ void k_renumber(const StepArgs a, const uint32_t* __restrict__ newid, uint32_t n2) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < n2; q += stride) {
        const uint32_t id = a.A.id[q];
        if (id >= a.n) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
        a.A.id[q] = newid[id];
    }
}

__global__ void k_compact_params(const StepArgs a, const uint8_t* __restrict__ alive, const uint32_t* __restrict__ newid,
                                 double* __restrict__ io) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        if (!alive[i]) continue;
        const uint32_t j = newid[i];
        io[j] = a.R64[i];
        io[np + j] = a.ccr64[i];
        io[2 * np + j] = a.cca64[i];
    }
}

// Order-preserving removal for batches: survivors of a.A go to a.B at dst[q]
// (exclusive prefix of the keep flags over the state order), so every
// replicate's cells stay one contiguous range; caller index newid[id].
__global__ void k_compact_state(const StepArgs a, const uint8_t* __restrict__ alive, const uint32_t* __restrict__ dst,
                                const uint32_t* __restrict__ newid) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = a.A.id[q];
        if (id >= a.n) {
            atomicOr(a.err, kErrIndex);
            continue;
        }
        if (!alive[id]) continue;
        const uint32_t f = dst[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a.B.pos64[d * np + f] = a.A.pos64[d * np + q];
            a.B.posf[d * np + f] = a.A.posf[d * np + q];
            a.B.comp[d * np + f] = a.A.comp[d * np + q];
            a.B.vp64[d * np + f] = a.A.vp64[d * np + q];
            a.B.vpf[d * np + f] = a.A.vpf[d * np + q];
        }
        a.B.rec[2 * (size_t)f] = a.A.rec[2 * (size_t)q];
        a.B.rec[2 * (size_t)f + 1] = a.A.rec[2 * (size_t)q + 1];
        a.B.id[f] = newid[id];
    }
}

// Additions to a batch: every cell of replicate r moves up by shift[r] (the
// cells added to the replicates before r), in state order (A -> B) and in
// caller order (its id and, into io, its FP64 parameters).
__global__ void k_shift_state(const StepArgs a, const uint32_t* __restrict__ shift) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t s = shift[rep_of_cell(a.grids, a.nrep, q)];
        const size_t f = (size_t)q + s;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a.B.pos64[d * np + f] = a.A.pos64[d * np + q];
            a.B.posf[d * np + f] = a.A.posf[d * np + q];
            a.B.comp[d * np + f] = a.A.comp[d * np + q];
            a.B.vp64[d * np + f] = a.A.vp64[d * np + q];
            a.B.vpf[d * np + f] = a.A.vpf[d * np + q];
        }
        a.B.rec[2 * f] = a.A.rec[2 * (size_t)q];
        a.B.rec[2 * f + 1] = a.A.rec[2 * (size_t)q + 1];
        a.B.id[f] = a.A.id[q] + s;  // a replicate's caller indices and slots span the same range
    }
}

__global__ void k_shift_params(const StepArgs a, const uint32_t* __restrict__ shift, double* __restrict__ io) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += stride) {
        const size_t j = (size_t)i + shift[rep_of_cell(a.grids, a.nrep, i)];
        io[j] = a.R64[i];
        io[np + j] = a.ccr64[i];
        io[2 * np + j] = a.cca64[i];
    }
}

// New cell k goes to slot and caller index dst[k]; io holds the m new
// positions (3 per cell) at io[0, 3m) and their R, ccr, cca at io[3m + k],
// io[4m + k], io[5m + k].
__global__ void k_append_state(const StepArgs a, const StateBuf st, const double* __restrict__ io,
                               const uint32_t* __restrict__ dst, const uint32_t* __restrict__ types, uint32_t m,
                               double* __restrict__ R64, double* __restrict__ ccr64, double* __restrict__ cca64) {
    const uint32_t stride = gridDim.x * blockDim.x;
    const size_t np = a.npad;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const size_t q = dst[j];
        if (q >= np) {  // the host computed every dst below the capacity
            atomicOr(a.err, kErrIndex);
            continue;
        }
        const double R = io[3 * (size_t)m + j], ccr = io[4 * (size_t)m + j], cca = io[5 * (size_t)m + j];
        R64[q] = R;
        ccr64[q] = ccr;
        cca64[q] = cca;
        // record: radius as FP32 plus its residual in units of ulp(R) / 2^11
        // (12 bits, offset 2^11) and the type, coefficient square roots; the
        // position fields are written by the next canonicalisation
        const float Rf = __double2float_rn(R);
        const uint32_t wzr = 0x8000u | radius_type_bits(R, Rf, types ? (types[j] & 15u) : 0u);
        st.rec[2 * q] = make_float4(0.f, 0.f, 0.f, Rf);
        st.rec[2 * q + 1] = make_float4(__double2float_rn(sqrt(ccr)), __double2float_rn(sqrt(cca)),
                                        __uint_as_float(0x80008000u), __uint_as_float(wzr));
        st.id[q] = (uint32_t)q;  // a new cell's caller index is its slot
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = io[3 * (size_t)j + d];
            const float xh = __double2float_rn(x);
            st.pos64[d * np + q] = x;
            st.posf[d * np + q] = xh;
            st.comp[d * np + q] = __double2float_rn(__dsub_rn((double)xh, x));
            st.vp64[d * np + q] = 0.0;
            st.vpf[d * np + q] = 0.0f;
        }
    }
}

__global__ void k_load_vprev(const StepArgs a, const StateBuf st, const double* __restrict__ in) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n; q += stride) {
        const uint32_t id = st.id[q];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double v = in ? in[3 * (size_t)id + d] : 0.0;
            if (a.mode == kFP64) st.vp64[(size_t)d * a.npad + q] = v;
            else st.vpf[(size_t)d * a.npad + q] = __double2float_rn(v);
        }
    }
}

int elementwise_grid(uint32_t n) {
    int g = (int)((n + 255u) / 256u);
    if (g < 1) g = 1;
    return std::min(g, device_sms() * 16);
}

}  // namespace

int device_sms() {
    constexpr int kMaxDev = 64;
    static std::atomic<int> cache[kMaxDev];  // 0 = not queried yet
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 152;
    int v = cache[dev].load(std::memory_order_relaxed);
    if (v > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 152;
    cache[dev].store(v, std::memory_order_relaxed);
    return v;
}

cudaError_t launch_zero_u32(uint32_t* p, size_t count, cudaStream_t s) {
    if (count == 0) return cudaSuccess;
    int g = (int)((count + 255) / 256);
    g = std::min(g, device_sms() * 32);
    k_zero_u32<<<g, 256, 0, s>>>(p, count);
    return cudaGetLastError();
}

cudaError_t launch_keys(const StepArgs& a, int grid, uint32_t vpad, cudaStream_t s) {
    if (a.n != 0) k_keys<<<grid, 256, 0, s>>>(a);
    // the scan's block sums of this histogram, by the reduce pass (per-warp
    // atomics into them from the key pass contend: consecutive warps of the
    // voxel-sorted cells hit the same 8,192-voxel block)
    k_scan_reduce<<<vpad / kScanTile, kScanThreads, 0, s>>>(a.count_cur, a.bcount_cur);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint32_t* count, uint32_t vpad, uint32_t* bsum, uint32_t* start, uint32_t* zero_word,
                        uint32_t* occ, cudaStream_t s) {
    const uint32_t nb = vpad / kScanTile;
    k_scan_reduce<<<nb, kScanThreads, 0, s>>>(count, bsum);
    k_scan_top<<<1, 1024, 0, s>>>(bsum, nb, zero_word);
    k_scan_down<<<nb, kScanThreads, 0, s>>>(count, bsum, start, reinterpret_cast<uint16_t*>(occ), nullptr);
    return cudaGetLastError();
}

cudaError_t launch_scan_blocks(const uint32_t* count, uint32_t vpad, uint32_t* bsum, uint32_t* zero_blocks,
                               uint32_t* start, uint32_t* zero_word, uint32_t* occ, cudaStream_t s) {
    const uint32_t nb = vpad / kScanTile;
    k_scan_top<<<1, 1024, 0, s>>>(bsum, nb, zero_word);
    k_scan_down<<<nb, kScanThreads, 0, s>>>(count, bsum, start, reinterpret_cast<uint16_t*>(occ), zero_blocks);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const StepArgs& a, int grid, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_scatter<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_canon(const StepArgs& a, int grid, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_canon<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_alive_flags(const uint8_t* alive, uint32_t n, uint32_t pad, uint32_t* flags, cudaStream_t s) {
    k_alive_flags<<<elementwise_grid(pad), 256, 0, s>>>(alive, n, pad, flags);
    return cudaGetLastError();
}

cudaError_t launch_keep_flags(const StepArgs& a, const StateBuf& st, const uint8_t* alive, uint32_t pad,
                              uint32_t* flags, cudaStream_t s) {
    k_keep_flags<<<elementwise_grid(pad), 256, 0, s>>>(a, st, alive, pad, flags);
    return cudaGetLastError();
}

cudaError_t launch_remove_in_place(const StepArgs& a, const uint8_t* alive, const uint32_t* keep_pref,
                                   const uint32_t* newid, uint32_t n2, uint32_t* hole, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const int g = elementwise_grid(a.n);
    k_list_holes<<<g, 256, 0, s>>>(a, alive, keep_pref, n2, hole);
    k_fill_holes<<<g, 256, 0, s>>>(a, alive, keep_pref, n2, hole);
    k_renumber<<<g, 256, 0, s>>>(a, newid, n2);
    return cudaGetLastError();
}

cudaError_t launch_compact_params(const StepArgs& a, const uint8_t* alive, const uint32_t* newid, double* io,
                                  cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_compact_params<<<elementwise_grid(a.n), 256, 0, s>>>(a, alive, newid, io);
    return cudaGetLastError();
}

cudaError_t launch_append_state(const StepArgs& a, const StateBuf& st, const double* io, const uint32_t* dst,
                                const uint32_t* types, uint32_t m, double* R64, double* ccr64, double* cca64,
                                cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    k_append_state<<<elementwise_grid(m), 256, 0, s>>>(a, st, io, dst, types, m, R64, ccr64, cca64);
    return cudaGetLastError();
}

cudaError_t launch_compact_state(const StepArgs& a, const uint8_t* alive, const uint32_t* dst, const uint32_t* newid,
                                 cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_compact_state<<<elementwise_grid(a.n), 256, 0, s>>>(a, alive, dst, newid);
    return cudaGetLastError();
}

cudaError_t launch_shift(const StepArgs& a, const uint32_t* shift, double* io, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_shift_state<<<elementwise_grid(a.n), 256, 0, s>>>(a, shift);
    k_shift_params<<<elementwise_grid(a.n), 256, 0, s>>>(a, shift, io);
    return cudaGetLastError();
}

size_t unpermute_scratch_bytes(uint32_t n) {
    const size_t nb = ((size_t)n + kUpIds - 1) >> kUpLog;
    return ((2 * (size_t)n + 255) / 256) * 256 + 4 * nb;
}

cudaError_t launch_unpermute_pos(const StepArgs& a, const StateBuf& st, double* out, double* stage, void* scratch,
                                 size_t scratch_cap, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    if (unpermute_scratch_bytes(a.n) > scratch_cap) return cudaErrorInvalidValue;
    const uint32_t nb = (a.n + kUpIds - 1) >> kUpLog;
    uint16_t* low = static_cast<uint16_t*>(scratch);
    uint32_t* cursor = reinterpret_cast<uint32_t*>(static_cast<char*>(scratch) + ((2 * (size_t)a.n + 255) / 256) * 256);
    cudaError_t e = cudaMemsetAsync(cursor, 0, 4 * (size_t)nb, s);
    if (e != cudaSuccess) return e;
    k_unpermute_pos_stage<<<elementwise_grid(a.n), 256, 0, s>>>(a, st, cursor, stage, low);
    k_unpermute_pos_place<<<nb, 256, 0, s>>>(a.n, stage, low, out);
    return cudaGetLastError();
}

cudaError_t launch_unpermute_vel(const StepArgs& a, const StateBuf& st, const float* vf, const double* vd,
                                 double* out, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_unpermute_vel<<<elementwise_grid(a.n), 256, 0, s>>>(a, st, vf, vd, out);
    return cudaGetLastError();
}

cudaError_t launch_load_pos(const StepArgs& a, const StateBuf& st, const double* in, int raw_kahan,
                            const double* comp_in, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_load_pos<<<elementwise_grid(a.n), 256, 0, s>>>(a, st, in, raw_kahan, comp_in);
    return cudaGetLastError();
}

cudaError_t launch_load_vprev(const StepArgs& a, const StateBuf& st, const double* in, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    k_load_vprev<<<elementwise_grid(a.n), 256, 0, s>>>(a, st, in);
    return cudaGetLastError();
}

}  // namespace mk
