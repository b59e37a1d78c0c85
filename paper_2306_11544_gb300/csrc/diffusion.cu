// Substrate diffusion-decay step and gradients on a voxel grid (the
// microenvironment solver and gradient regions of Sec. 5.1-5.2: a 75^3-voxel
// domain in the paper's runs).  The paper gives no numerical method; the
// statement implemented:
//
//   S densities rho_s on nx x ny x nz cubic voxels of side dx (voxel
//   v = x + nx (y + ny z), array [s][v]), diffusion coefficient D_s, decay
//   lambda_s, no flux through the faces.  A step of length dt is three
//   one-dimensional backward-Euler solves, along x, then y, then z, the decay
//   shared equally: along a line of n voxels, with k = D dt / dx^2 and
//   e = lambda dt / 3, the tridiagonal system has diagonal 1 + 2k + e inside,
//   1 + k + e at the two faces (a mirrored neighbour: no flux), 1 + e for
//   n = 1, and off-diagonals -k.  It is solved by Gaussian elimination
//   without pivoting (the Thomas algorithm), with coefficients shared by all
//   lines of an axis and the pivots inverted once:
//      m_0 = T_00;  m_i = T_ii + k c_{i-1} (i >= 1);  w_i = 1 / m_i;
//      c_i = -k w_i
//   (no division inside the recurrences), in its two-ended form: the matrix
//   reads the same from either end (T_ii = T_{n-1-i,n-1-i}), so eliminating
//   upward from the last row produces the same pivots in mirror order, bit
//   for bit.  With p = floor(n / 2):
//      top    y_0 = old_0 w_0;  y_i = (old_i + k y_{i-1}) w_i        (i < p)
//      bottom z_{n-1} = old_{n-1} w_0;
//             z_i = (old_i + k z_{i+1}) w_{n-1-i}                  (i > p)
//      meet   u_p = ((old_p + k y_{p-1}) + k z_{p+1}) / g,
//             g = T_pp + k c_{p-1} + k c_{n-2-p}
//             (a term is absent when its row is: p = 0, or p = n - 1)
//      back   u_i = y_i - c_i u_{i+1} (i = p-1 .. 0);
//             u_i = z_i - c_{n-1-i} u_{i-1} (i = p+1 .. n-1)
//   The solution is that of the one-ended elimination up to rounding, and a
//   line's dependent chain is n steps instead of 2 n: two threads share a
//   line, one per end.  Arithmetic: FP64, each a + b c above one fused
//   multiply-add (three FP64 operations per value and solve: this GPU's FP64
//   pipe runs at about 1/60 of its FP32 rate, and it, not memory, bounds the
//   solver), IEEE operations in a fixed order, so every value is
//   reproducible run to run.  Gradients: central differences inside,
//   one-sided at the faces, zero along an axis of one voxel, each difference
//   times the reciprocal of dx or 2 dx; array [s][axis][v].
//
// GB300 mapping: the work is a set of independent recurrences (one per end
// of a grid line), so every kernel runs two threads per line.  Lines along y
// and z are strided in memory but their neighbours along x are adjacent: a
// warp takes 16 adjacent lines, lanes 0-15 their top ends and lanes 16-31
// their bottom ends, so every step of the recurrence is two coalesced
// 128-byte accesses, and the two ends meet through one shuffle.  Lines along
// x are contiguous, so a block of two warps first stages 32 lines (one
// contiguous run of memory) in shared memory with coalesced loads; warp 0
// solves their top ends and warp 1 their bottom ends there, and the block
// writes them back.  A 75^3 field of a few substrates (3.4 MB each) stays in
// L2 between the three solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "mech.h"
#include "mech_internal.cuh"

#define DTRY(expr)                      \
    do {                                \
        const int rc_ = (expr);         \
        if (rc_ != MECH_OK) return rc_; \
    } while (0)

namespace {

constexpr int kLineTile = 32;   // x lines staged per block (two warps: one per line end)
constexpr int kMaxNxTile = 189;  // 32 lines of up to 189 doubles (odd stride) and the meeting values fit in 48 KB
constexpr int kLinesPerWarp = 16;  // y/z and long x lines: 16 lines per warp, both ends

// Diagonal entry i of the tridiagonal matrix of a line of n voxels.
__device__ __forceinline__ double diag_entry(int64_t i, int64_t n, double k, double e) {
    if (n == 1) return __dadd_rn(1.0, e);
    if (i == 0 || i == n - 1) return __dadd_rn(__dadd_rn(1.0, k), e);
    return __dadd_rn(__dadd_rn(1.0, __dmul_rn(2.0, k)), e);
}

// Coefficients of one (substrate, axis) pair t = 3 s + axis: reciprocal
// pivots w (in m) and c, nmax each; the reciprocal of the meeting row's pivot
// g (in gi); and k per substrate.
__device__ __forceinline__ void coeffs_one(int64_t t, int64_t nx, int64_t ny, int64_t nz, int64_t nmax, double dx,
                                           double dt, const double* __restrict__ D, const double* __restrict__ lam,
                                           double* __restrict__ m, double* __restrict__ c, double* __restrict__ gi,
                                           double* __restrict__ kk) {
    const int64_t s = t / 3, a = t - 3 * s;
    const int64_t n = a == 0 ? nx : (a == 1 ? ny : nz);
    const double k = __ddiv_rn(__dmul_rn(D[s], dt), __dmul_rn(dx, dx));
    const double e = __ddiv_rn(__dmul_rn(lam[s], dt), 3.0);
    if (a == 0) kk[s] = k;
    double* mm = m + (size_t)t * nmax;
    double* cc = c + (size_t)t * nmax;
    for (int64_t i = 0; i < n; ++i) {
        const double diag = diag_entry(i, n, k, e);
        const double piv = i == 0 ? diag : __dadd_rn(diag, __dmul_rn(k, cc[i - 1]));
        mm[i] = __ddiv_rn(1.0, piv);
        if (i < n - 1) cc[i] = __dmul_rn(-k, mm[i]);
    }
    const int64_t p = n >> 1;
    double g = diag_entry(p, n, k, e);
    if (p >= 1) g = __dadd_rn(g, __dmul_rn(k, cc[p - 1]));
    if (p <= n - 2) g = __dadd_rn(g, __dmul_rn(k, cc[n - 2 - p]));
    gi[t] = __ddiv_rn(1.0, g);
}

// Coefficients of every (substrate, axis): a grid-stride loop over the 3 S
// (substrate, axis) pairs, one thread each.
__global__ void k_diff_coeffs(int32_t S, int64_t nx, int64_t ny, int64_t nz, int64_t nmax, double dx, double dt,
                              const double* __restrict__ D, const double* __restrict__ lam, double* __restrict__ m,
                              double* __restrict__ c, double* __restrict__ gi, double* __restrict__ kk) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 3 * (int64_t)S;
         t += (int64_t)gridDim.x * blockDim.x)
        coeffs_one(t, nx, ny, nz, nmax, dx, dt, D, lam, m, c, gi, kk);
}

// One end of a line of n values (any memory space): the top end is rows
// 0 .. p-1 from base = row 0 with step +stride, the bottom end rows
// n-1 .. p+1 from base = row n-1 with step -stride; row j of an end (j-th
// from its extremity) has pivot w_j and back coefficient c_j.
struct LineEnd {
    double* base;
    int64_t step;
    int64_t cnt;  // rows of this end: p (top) or n - 1 - p (bottom)
};

__device__ __forceinline__ LineEnd line_end(double* row0, int64_t stride, int64_t n, bool top) {
    const int64_t p = n >> 1;
    return top ? LineEnd{row0, stride, p} : LineEnd{row0 + (n - 1) * stride, -stride, n - 1 - p};
}

// Elimination toward the meeting row; returns the last value (0 without rows).
__device__ __forceinline__ double end_eliminate(const LineEnd& L, double k, const double* __restrict__ w) {
    double prev = 0.0;
    for (int64_t j = 0; j < L.cnt; ++j) {
        const double r = L.base[j * L.step];
        prev = j == 0 ? __dmul_rn(r, w[0]) : __dmul_rn(__fma_rn(k, prev, r), w[j]);
        L.base[j * L.step] = prev;
    }
    return prev;
}

// Value of the meeting row from its right-hand side and the two ends' last values.
__device__ __forceinline__ double meet(double rp, double k, double y, double z, double gi) {
    return __dmul_rn(__fma_rn(k, z, __fma_rn(k, y, rp)), gi);
}

// Back substitution from the meeting row out to the end's extremity.
__device__ __forceinline__ void end_back(const LineEnd& L, const double* __restrict__ c, double up) {
    double next = up;
    for (int64_t j = L.cnt - 1; j >= 0; --j) {
        next = __fma_rn(-c[j], next, L.base[j * L.step]);
        L.base[j * L.step] = next;
    }
}

// The same two recurrences with the whole end in registers (cnt <= MAXC):
// all its values are loaded in one round before the elimination starts (the
// loop above waits for every load in turn), only the solution is stored.
template <int MAXC>
__device__ __forceinline__ double regs_eliminate(const LineEnd& L, double k, const double* __restrict__ w,
                                                 double (&v)[MAXC]) {
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j < L.cnt) v[j] = L.base[j * L.step];
    double prev = 0.0;
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j < L.cnt) {
            prev = j == 0 ? __dmul_rn(v[0], w[0]) : __dmul_rn(__fma_rn(k, prev, v[j]), w[j]);
            v[j] = prev;
        }
    return prev;
}

template <int MAXC>
__device__ __forceinline__ void regs_back(const LineEnd& L, const double* __restrict__ c, double up,
                                          double (&v)[MAXC]) {
    double next = up;
#pragma unroll
    for (int j = MAXC - 1; j >= 0; --j)
        if (j < L.cnt) {
            next = __fma_rn(-c[j], next, v[j]);
            v[j] = next;
        }
#pragma unroll
    for (int j = 0; j < MAXC; ++j)
        if (j < L.cnt) L.base[j * L.step] = v[j];
}

// Register capacity for a line of n values: each end holds at most n / 2.
constexpr int kRegsSmall = 16, kRegsLarge = 40;
inline int regs_for(int64_t n) { return n <= 2 * kRegsSmall + 1 ? kRegsSmall : (n <= 2 * kRegsLarge + 1 ? kRegsLarge : 0); }

// x lines: line L = (s nz + z) ny + y occupies rho[L nx, (L + 1) nx).  A
// block stages lines [L0, L0 + 32) (one contiguous run) in shared memory;
// thread (line l = tid mod 32, end = tid / 32) solves one end of line l, the
// ends meet through shared memory, and the block writes the lines back.  The
// shared row stride is odd (in doubles), so the 16 lanes of a half-warp hit
// 16 different banks.  MAXC > 0: a line end (at most MAXC values) is solved
// in registers; the launch bound caps registers so that six blocks fit on
// an SM (the 75^3 grid's 704 blocks then run in one wave).
template <int MAXC>
__global__ void __launch_bounds__(2 * kLineTile, 6) k_diff_x_tiled(double* __restrict__ rho, int64_t lines, int64_t nx,
                                                               int64_t ny, int64_t nz, int64_t nmax,
                                                               const double* __restrict__ m,
                                                               const double* __restrict__ c,
                                                               const double* __restrict__ gi,
                                                               const double* __restrict__ kk) {
    extern __shared__ double tile[];
    __shared__ double s_last[2 * kLineTile];
    const int64_t stride = nx | 1;
    const int l = threadIdx.x & (kLineTile - 1);
    const bool top = threadIdx.x < kLineTile;
    const int64_t p = nx >> 1;
    // element w of a staged run is (line w / nx, column w % nx), tile slot
    // line * stride + column; a run holds at most 32 x 189 values, so the
    // copies use 32-bit indices advanced by 64 = dr lines + dc columns
    // without a division
    const uint32_t n32 = (uint32_t)nx, st32 = (uint32_t)stride;
    const uint32_t dr = (2u * kLineTile) / n32, dc = (2u * kLineTile) - dr * n32;
    const uint32_t r0 = threadIdx.x / n32, c0 = threadIdx.x - r0 * n32;
    auto copy = [&](double* run, bool to_tile, uint32_t W) {
        uint32_t r = r0, col = c0;
        for (uint32_t w = threadIdx.x; w < W; w += 2u * kLineTile) {
            if (to_tile) tile[r * st32 + col] = run[w];
            else run[w] = tile[r * st32 + col];
            r += dr;
            col += dc;
            if (col >= n32) {
                col -= n32;
                ++r;
            }
        }
    };
    for (int64_t L0 = (int64_t)blockIdx.x * kLineTile; L0 < lines; L0 += (int64_t)gridDim.x * kLineTile) {
        const int64_t cnt = lines - L0 < kLineTile ? lines - L0 : kLineTile;
        const uint32_t W = (uint32_t)(cnt * nx);
        copy(rho + L0 * nx, true, W);
        __syncthreads();
        const int64_t s = (L0 + l) / (ny * nz);
        double* row = tile + l * stride;
        const LineEnd end = line_end(row, 1, nx, top);
        double rp = 0.0;
        double v[MAXC > 0 ? MAXC : 1];
        if (l < cnt) {
            rp = row[p];  // read by both ends before either writes it
            const double* w = m + (size_t)(3 * s) * nmax;
            if constexpr (MAXC > 0) s_last[threadIdx.x] = regs_eliminate<MAXC>(end, kk[s], w, v);
            else s_last[threadIdx.x] = end_eliminate(end, kk[s], w);
        }
        __syncthreads();
        if (l < cnt) {
            const double up = meet(rp, kk[s], s_last[l], s_last[kLineTile + l], gi[3 * s]);
            const double* cc = c + (size_t)(3 * s) * nmax;
            if constexpr (MAXC > 0) regs_back<MAXC>(end, cc, up, v);
            else end_back(end, cc, up);
            if (top) row[p] = up;
        }
        __syncthreads();
        copy(rho + L0 * nx, false, W);
        __syncthreads();
    }
}

// Lines of n values at rho + base(L), stride apart, two lanes per line: a
// warp takes lines [L0, L0 + 16), lanes 0-15 their top ends and lanes 16-31
// their bottom ends (lane pairs l, l + 16 share a line), and the ends meet
// through one shuffle.  The loop runs per warp, so every lane reaches the
// shuffle.  base(L) and the coefficient row t(L) come from the functor.
template <int MAXC, typename Line>
__device__ __forceinline__ void solve_lines_by_warp(double* __restrict__ rho, int64_t lines, int64_t n,
                                                    int64_t stride, int64_t nmax, const double* __restrict__ m,
                                                    const double* __restrict__ c, const double* __restrict__ gi,
                                                    const double* __restrict__ kk, Line line) {
    const int lane = threadIdx.x & 31;
    const bool top = lane < kLinesPerWarp;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t p = n >> 1;
    for (int64_t L0 = warp * kLinesPerWarp; L0 < lines; L0 += nwarps * kLinesPerWarp) {
        const int64_t L = L0 + (lane & (kLinesPerWarp - 1));
        const bool valid = L < lines;
        int64_t base = 0, s = 0, t = 0;
        if (valid) line(L, base, s, t);
        double* row0 = rho + base;
        const LineEnd end = line_end(row0, stride, n, top);
        double rp = 0.0, last = 0.0;
        double v[MAXC > 0 ? MAXC : 1];
        if (valid) {
            rp = row0[p * stride];  // read by both ends before either writes it
            if constexpr (MAXC > 0) last = regs_eliminate<MAXC>(end, kk[s], m + (size_t)t * nmax, v);
            else last = end_eliminate(end, kk[s], m + (size_t)t * nmax);
        }
        const double other = __shfl_xor_sync(0xFFFFFFFFu, last, kLinesPerWarp);
        __syncwarp();  // orders the reads of row p above before its write below
        if (valid) {
            const double up = meet(rp, kk[s], top ? last : other, top ? other : last, gi[t]);
            if constexpr (MAXC > 0) regs_back<MAXC>(end, c + (size_t)t * nmax, up, v);
            else end_back(end, c + (size_t)t * nmax, up);
            if (top) row0[p * stride] = up;
        }
    }
}

// x lines longer than a shared-memory tile allows (and than the register
// form holds): walked in global memory.
__global__ void k_diff_x_direct(double* __restrict__ rho, int64_t lines, int64_t nx, int64_t ny, int64_t nz,
                                int64_t nmax, const double* __restrict__ m, const double* __restrict__ c,
                                const double* __restrict__ gi, const double* __restrict__ kk) {
    solve_lines_by_warp<0>(rho, lines, nx, 1, nmax, m, c, gi, kk,
                           [&](int64_t L, int64_t& base, int64_t& s, int64_t& t) {
                               s = L / (ny * nz);
                               base = L * nx;
                               t = 3 * s;
                           });
}

// y lines (axis 1) or z lines (axis 2): line L = (s, outer, x), consecutive
// lines are consecutive x, so every step of the recurrence is coalesced.
template <int MAXC>
__global__ void k_diff_yz(double* __restrict__ rho, int axis, int32_t S, int64_t nx, int64_t ny, int64_t nz,
                          int64_t nmax, const double* __restrict__ m, const double* __restrict__ c,
                          const double* __restrict__ gi, const double* __restrict__ kk) {
    const int64_t nv = nx * ny * nz;
    const int64_t outer = axis == 1 ? nz : ny;
    const int64_t lines = (int64_t)S * outer * nx;
    const int64_t n = axis == 1 ? ny : nz;
    const int64_t stride = axis == 1 ? nx : nx * ny;
    solve_lines_by_warp<MAXC>(rho, lines, n, stride, nmax, m, c, gi, kk,
                        [&](int64_t L, int64_t& base, int64_t& s, int64_t& t) {
                            const int64_t x = L % nx;
                            const int64_t r = L / nx;
                            const int64_t o = r % outer;
                            s = r / outer;
                            base = s * nv + x + (axis == 1 ? o * nx * ny : o * nx);
                            t = 3 * s + axis;
                        });
}

// Gradients, one thread per (substrate, voxel) value: differences divided
// by dx or 2 dx as products with their reciprocals (formed once on the host:
// an FP64 division costs about six FP64 additions here), and 32-bit index
// arithmetic (at most 4e9 values per handle).
__global__ void k_diff_gradient(const double* __restrict__ rho, int32_t S, uint32_t nx, uint32_t ny, uint32_t nz,
                                double inv_dx, double inv_2dx, double* __restrict__ grad) {
    const uint32_t nxy = nx * ny, nv = nxy * nz;
    const uint32_t total = (uint32_t)S * nv;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
        const uint32_t s = t / nv, v = t - s * nv;
        const uint32_t z = v / nxy, rem = v - z * nxy;
        const uint32_t y = rem / nx, x = rem - y * nx;
        const double* r = rho + (size_t)s * nv;
        const uint32_t n[3] = {nx, ny, nz};
        const uint32_t i[3] = {x, y, z};
        const uint32_t st[3] = {1u, nx, nxy};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double g;
            if (n[a] == 1u) g = 0.0;
            else if (i[a] == 0u) g = __dmul_rn(__dsub_rn(r[v + st[a]], r[v]), inv_dx);
            else if (i[a] == n[a] - 1u) g = __dmul_rn(__dsub_rn(r[v], r[v - st[a]]), inv_dx);
            else g = __dmul_rn(__dsub_rn(r[v + st[a]], r[v - st[a]]), inv_2dx);
            grad[((size_t)s * 3 + a) * nv + v] = g;
        }
    }
}

int grid_for(int64_t work, int block, int sms) {
    int64_t g = (work + block - 1) / block;
    const int64_t cap = (int64_t)sms * 32;
    if (g > cap) g = cap;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

struct mech_diffusion {
    int dev = 0;
    int sms = 152;
    cudaStream_t own_stream = nullptr;
    cudaStream_t stream = nullptr;
    int64_t nx = 0, ny = 0, nz = 0, nv = 0, nmax = 0;
    int32_t S = 0;
    double dx = 0.0;
    double dt_coef = -1.0;  // dt of the current coefficients (none yet)
    double* d_rho = nullptr;
    double* d_grad = nullptr;
    double* d_D = nullptr;
    double* d_lam = nullptr;
    double* d_m = nullptr;
    double* d_c = nullptr;
    double* d_gi = nullptr;
    double* d_k = nullptr;
    std::vector<void*> allocs;

    ~mech_diffusion() {
        for (void* p : allocs) cudaFree(p);
        if (own_stream) cudaStreamDestroy(own_stream);
    }
    template <typename T>
    int alloc(T** p, size_t count) {
        void* q = nullptr;
        const cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return mk::record_error(MECH_E_OOM, std::string("mech_diffusion: cudaMalloc failed: ") +
                                                    cudaGetErrorString(e));
        }
        allocs.push_back(q);
        *p = static_cast<T*>(q);
        return MECH_OK;
    }
};

namespace {

int dcheck(mech_diffusion_t* h) {
    return h ? MECH_OK : mk::record_error(MECH_E_ARG, "null diffusion handle");
}

int dcuda(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return MECH_OK;
    cudaGetLastError();
    return mk::record_error(MECH_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace

extern "C" {

int mech_diffusion_create(mech_diffusion_t** out, int64_t nx, int64_t ny, int64_t nz, int32_t n_substrates,
                          double dx, const double* D, const double* lambda) {
    if (!out) return mk::record_error(MECH_E_ARG, "null output handle");
    *out = nullptr;
    if (nx < 1 || ny < 1 || nz < 1 || n_substrates < 1)
        return mk::record_error(MECH_E_ARG, "grid sizes and the substrate count must be >= 1");
    if ((double)nx * (double)ny * (double)nz * (double)n_substrates > 4.0e9)
        return mk::record_error(MECH_E_ARG, "more than 4e9 voxel values");
    if (!(dx > 0.0) || !std::isfinite(dx)) return mk::record_error(MECH_E_ARG, "dx must be positive and finite");
    if (!D || !lambda) return mk::record_error(MECH_E_ARG, "null coefficient array");
    for (int32_t s = 0; s < n_substrates; ++s)
        if (!(D[s] >= 0.0) || !(lambda[s] >= 0.0) || !std::isfinite(D[s]) || !std::isfinite(lambda[s]))
            return mk::record_error(MECH_E_ARG, "D and lambda must be finite and >= 0");
    auto* h = new mech_diffusion();
    auto bail = [&](int rc) {
        delete h;
        return rc;
    };
    int rc = dcuda(cudaGetDevice(&h->dev), "cudaGetDevice");
    if (rc != MECH_OK) return bail(rc);
    int sms = 0;
    rc = dcuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->dev), "cudaDeviceGetAttribute");
    if (rc != MECH_OK) return bail(rc);
    h->sms = sms;
    rc = dcuda(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking), "cudaStreamCreate");
    if (rc != MECH_OK) return bail(rc);
    h->stream = h->own_stream;
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->nv = nx * ny * nz;
    h->nmax = std::max(nx, std::max(ny, nz));
    h->S = n_substrates;
    h->dx = dx;
    const size_t nvals = (size_t)h->nv * (size_t)h->S;
    rc = h->alloc(&h->d_rho, nvals);
    if (rc == MECH_OK) rc = h->alloc(&h->d_grad, 3 * nvals);
    if (rc == MECH_OK) rc = h->alloc(&h->d_D, (size_t)h->S);
    if (rc == MECH_OK) rc = h->alloc(&h->d_lam, (size_t)h->S);
    if (rc == MECH_OK) rc = h->alloc(&h->d_m, (size_t)3 * h->S * h->nmax);
    if (rc == MECH_OK) rc = h->alloc(&h->d_c, (size_t)3 * h->S * h->nmax);
    if (rc == MECH_OK) rc = h->alloc(&h->d_gi, (size_t)3 * h->S);
    if (rc == MECH_OK) rc = h->alloc(&h->d_k, (size_t)h->S);
    if (rc != MECH_OK) return bail(rc);
    rc = dcuda(cudaMemcpyAsync(h->d_D, D, h->S * 8, cudaMemcpyHostToDevice, h->stream), "upload D");
    if (rc == MECH_OK) rc = dcuda(cudaMemcpyAsync(h->d_lam, lambda, h->S * 8, cudaMemcpyHostToDevice, h->stream),
                                  "upload lambda");
    if (rc == MECH_OK) rc = dcuda(cudaMemsetAsync(h->d_rho, 0, nvals * 8, h->stream), "zero densities");
    if (rc == MECH_OK) rc = dcuda(cudaStreamSynchronize(h->stream), "create");
    if (rc != MECH_OK) return bail(rc);
    // the staged x tile needs at most 32 x 189 doubles = 48,384 bytes, and the
    // meeting values 512 bytes, within the default 48 KiB of shared memory: no
    // per-function attribute (a process-wide setting) is changed
    static_assert((kLineTile * (kMaxNxTile | 1) + 2 * kLineTile) * sizeof(double) <= 48 * 1024,
                  "x tile and meeting values within the default limit");
    *out = h;
    return MECH_OK;
}

int mech_diffusion_destroy(mech_diffusion_t* h) {
    if (!h) return MECH_OK;
    cudaStreamSynchronize(h->stream);
    delete h;
    return MECH_OK;
}

int mech_diffusion_set_stream(mech_diffusion_t* h, void* stream) {
    DTRY(dcheck(h));
    cudaStreamSynchronize(h->stream);
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return MECH_OK;
}

int mech_diffusion_write(mech_diffusion_t* h, const double* rho) {
    DTRY(dcheck(h));
    if (!rho) return mk::record_error(MECH_E_ARG, "null densities");
    const size_t n = (size_t)h->nv * h->S;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(rho[i])) return mk::record_error(MECH_E_NONFINITE, "non-finite density");
    DTRY(dcuda(cudaMemcpyAsync(h->d_rho, rho, n * 8, cudaMemcpyHostToDevice, h->stream), "write densities"));
    return dcuda(cudaStreamSynchronize(h->stream), "write densities");
}

int mech_diffusion_read(mech_diffusion_t* h, double* rho) {
    DTRY(dcheck(h));
    if (!rho) return mk::record_error(MECH_E_ARG, "null output");
    DTRY(dcuda(cudaMemcpyAsync(rho, h->d_rho, (size_t)h->nv * h->S * 8, cudaMemcpyDeviceToHost, h->stream),
                   "read densities"));
    return dcuda(cudaStreamSynchronize(h->stream), "read densities");
}

int mech_diffusion_step(mech_diffusion_t* h, double dt, int64_t n_steps) {
    DTRY(dcheck(h));
    if (!(dt >= 0.0) || !std::isfinite(dt)) return mk::record_error(MECH_E_ARG, "dt must be finite and >= 0");
    if (n_steps < 0) return mk::record_error(MECH_E_ARG, "negative step count");
    if (n_steps == 0) return MECH_OK;
    if (dt != h->dt_coef) {
        k_diff_coeffs<<<grid_for(3 * h->S, 64, h->sms), 64, 0, h->stream>>>(h->S, h->nx, h->ny, h->nz, h->nmax,
                                                                               h->dx, dt, h->d_D, h->d_lam, h->d_m,
                                                                               h->d_c, h->d_gi, h->d_k);
        DTRY(dcuda(cudaGetLastError(), "coefficients"));
        h->dt_coef = dt;
    }
    const int64_t xlines = (int64_t)h->S * h->ny * h->nz;
    const int64_t ylines = (int64_t)h->S * h->nz * h->nx;
    const int64_t zlines = (int64_t)h->S * h->ny * h->nx;
    // two threads per line everywhere: 32 staged x lines per 64-thread block,
    // otherwise 16 lines per warp
    const int xblocks = grid_for(xlines, kLineTile, h->sms);
    const int xbytes = (int)(kLineTile * (h->nx | 1) * sizeof(double));
    const int wblock = 128, lines_per_block = wblock / 32 * kLinesPerWarp;
    const int rx = regs_for(h->nx), ry = regs_for(h->ny), rz = regs_for(h->nz);
    for (int64_t step = 0; step < n_steps; ++step) {
        if (h->nx <= kMaxNxTile) {
            auto kx = rx == kRegsSmall ? k_diff_x_tiled<kRegsSmall>
                                       : (rx == kRegsLarge ? k_diff_x_tiled<kRegsLarge> : k_diff_x_tiled<0>);
            kx<<<xblocks, 2 * kLineTile, xbytes, h->stream>>>(h->d_rho, xlines, h->nx, h->ny, h->nz, h->nmax,
                                                              h->d_m, h->d_c, h->d_gi, h->d_k);
        } else {
            k_diff_x_direct<<<grid_for(xlines, lines_per_block, h->sms), wblock, 0, h->stream>>>(
                h->d_rho, xlines, h->nx, h->ny, h->nz, h->nmax, h->d_m, h->d_c, h->d_gi, h->d_k);
        }
        for (int axis = 1; axis <= 2; ++axis) {
            const int r = axis == 1 ? ry : rz;
            auto ky = r == kRegsSmall ? k_diff_yz<kRegsSmall> : (r == kRegsLarge ? k_diff_yz<kRegsLarge> : k_diff_yz<0>);
            ky<<<grid_for(axis == 1 ? ylines : zlines, lines_per_block, h->sms), wblock, 0, h->stream>>>(
                h->d_rho, axis, h->S, h->nx, h->ny, h->nz, h->nmax, h->d_m, h->d_c, h->d_gi, h->d_k);
        }
        DTRY(dcuda(cudaGetLastError(), "diffusion step"));
    }
    return MECH_OK;
}

int mech_diffusion_gradient(mech_diffusion_t* h, double* grad) {
    DTRY(dcheck(h));
    k_diff_gradient<<<grid_for((int64_t)h->S * h->nv, 256, h->sms), 256, 0, h->stream>>>(
        h->d_rho, h->S, (uint32_t)h->nx, (uint32_t)h->ny, (uint32_t)h->nz, 1.0 / h->dx, 0.5 / h->dx, h->d_grad);
    DTRY(dcuda(cudaGetLastError(), "gradient"));
    if (grad)
        DTRY(dcuda(cudaMemcpyAsync(grad, h->d_grad, (size_t)3 * h->nv * h->S * 8, cudaMemcpyDeviceToHost,
                                       h->stream),
                       "read gradients"));
    return dcuda(cudaStreamSynchronize(h->stream), "gradient");
}

int mech_diffusion_sync(mech_diffusion_t* h) {
    DTRY(dcheck(h));
    return dcuda(cudaStreamSynchronize(h->stream), "sync");
}

}  // extern "C"
