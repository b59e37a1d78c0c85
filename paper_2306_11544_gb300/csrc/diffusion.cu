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
//   n = 1, and off-diagonals -k.  It is solved by the Thomas algorithm with
//   coefficients shared by all lines of an axis, the pivots inverted once:
//      m_0 = T_00;  m_i = T_ii + k c_{i-1} (i >= 1);  w_i = 1 / m_i;
//      c_i = -k w_i
//      forward  r_0 = old_0 w_0;  r_i = (old_i + k r_{i-1}) w_i
//      backward r_i = r_i - c_i r_{i+1}   (i = n-2 .. 0)
//   (no division inside the recurrences: an FP64 division costs about six
//   FP64 additions on this GPU; the plain elimination divides by m_i, and the
//   two arrangements agree to rounding), in FP64 with IEEE operations in this
//   order (no contraction), so every value is reproducible run to run.  Gradients: central differences inside, one-sided
//   at the faces, zero along an axis of one voxel; array [s][axis][v].
//
// GB300 mapping: the work is a set of independent recurrences (one per grid
// line), so every kernel runs one thread per line.  Lines along y and z are
// strided in memory but their neighbours along x are adjacent, so a warp's 32
// lines make coalesced accesses at every step of the recurrence.  Lines along
// x are contiguous, so a warp first stages its 32 lines (one contiguous run of
// memory) in shared memory with coalesced loads, solves there, and writes them
// back.  A 75^3 field of a few substrates (3.4 MB each) stays in L2 between
// the three solves.
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

constexpr int kLineTile = 32;   // x lines staged per warp
constexpr int kMaxNxTile = 191;  // 32 lines of up to 191 doubles (+1 pad) fit in 48 KB of shared memory

// Thomas coefficients of one (substrate, axis) pair t = 3 s + axis.
__device__ __forceinline__ void coeffs_one(int64_t t, int64_t nx, int64_t ny, int64_t nz, int64_t nmax, double dx,
                                           double dt, const double* __restrict__ D, const double* __restrict__ lam,
                                           double* __restrict__ m, double* __restrict__ c, double* __restrict__ kk) {
    const int64_t s = t / 3, a = t - 3 * s;
    const int64_t n = a == 0 ? nx : (a == 1 ? ny : nz);
    const double k = __ddiv_rn(__dmul_rn(D[s], dt), __dmul_rn(dx, dx));
    const double e = __ddiv_rn(__dmul_rn(lam[s], dt), 3.0);
    if (a == 0) kk[s] = k;
    double* mm = m + (size_t)t * nmax;
    double* cc = c + (size_t)t * nmax;
    for (int64_t i = 0; i < n; ++i) {
        double diag;
        if (n == 1) diag = __dadd_rn(1.0, e);
        else if (i == 0 || i == n - 1) diag = __dadd_rn(__dadd_rn(1.0, k), e);
        else diag = __dadd_rn(__dadd_rn(1.0, __dmul_rn(2.0, k)), e);
        const double piv = i == 0 ? diag : __dadd_rn(diag, __dmul_rn(k, cc[i - 1]));
        mm[i] = __ddiv_rn(1.0, piv);
        if (i < n - 1) cc[i] = __dmul_rn(-k, mm[i]);
    }
}

// Thomas coefficients of every (substrate, axis): reciprocal pivots w (in m)
// and c, nmax each; and k per substrate.  A grid-stride loop over the 3 S
// (substrate, axis) pairs, one thread each.
__global__ void k_diff_coeffs(int32_t S, int64_t nx, int64_t ny, int64_t nz, int64_t nmax, double dx, double dt,
                              const double* __restrict__ D, const double* __restrict__ lam, double* __restrict__ m,
                              double* __restrict__ c, double* __restrict__ kk) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < 3 * (int64_t)S;
         t += (int64_t)gridDim.x * blockDim.x)
        coeffs_one(t, nx, ny, nz, nmax, dx, dt, D, lam, m, c, kk);
}

// One line of n values at p[0], p[stride], ... in place (any memory space);
// w holds the reciprocal pivots.
__device__ __forceinline__ void thomas(double* p, int64_t stride, int64_t n, double k, const double* __restrict__ w,
                                       const double* __restrict__ c) {
    double prev = __dmul_rn(p[0], w[0]);
    p[0] = prev;
    for (int64_t i = 1; i < n; ++i) {
        prev = __dmul_rn(__dadd_rn(p[i * stride], __dmul_rn(k, prev)), w[i]);
        p[i * stride] = prev;
    }
    double next = prev;
    for (int64_t i = n - 2; i >= 0; --i) {
        next = __dsub_rn(p[i * stride], __dmul_rn(c[i], next));
        p[i * stride] = next;
    }
}

// x lines: line L = (s nz + z) ny + y occupies rho[L nx, (L + 1) nx).  A warp
// stages lines [L0, L0 + 32) (one contiguous run) in shared memory, each lane
// solves one, and the warp writes them back.  The shared row stride is odd
// (in doubles), so the 16 lanes of a half-warp hit 16 different banks.
__global__ void __launch_bounds__(kLineTile) k_diff_x_tiled(double* __restrict__ rho, int64_t lines, int64_t nx,
                                                           int64_t ny, int64_t nz, int64_t nmax,
                                                           const double* __restrict__ m, const double* __restrict__ c,
                                                           const double* __restrict__ kk) {
    extern __shared__ double tile[];
    const int64_t stride = nx | 1;
    const int lane = threadIdx.x;
    for (int64_t L0 = (int64_t)blockIdx.x * kLineTile; L0 < lines; L0 += (int64_t)gridDim.x * kLineTile) {
        const int64_t cnt = lines - L0 < kLineTile ? lines - L0 : kLineTile;
        const double* src = rho + L0 * nx;
        for (int64_t w = lane; w < cnt * nx; w += kLineTile) tile[(w / nx) * stride + w % nx] = src[w];
        __syncwarp();
        if (lane < cnt) {
            const int64_t L = L0 + lane;
            const int64_t s = L / (ny * nz);
            thomas(tile + lane * stride, 1, nx, kk[s], m + (size_t)(3 * s) * nmax, c + (size_t)(3 * s) * nmax);
        }
        __syncwarp();
        double* dst = rho + L0 * nx;
        for (int64_t w = lane; w < cnt * nx; w += kLineTile) dst[w] = tile[(w / nx) * stride + w % nx];
        __syncwarp();
    }
}

// x lines longer than a shared-memory tile allows: each thread walks its own line.
__global__ void k_diff_x_direct(double* __restrict__ rho, int64_t lines, int64_t nx, int64_t ny, int64_t nz,
                                int64_t nmax, const double* __restrict__ m, const double* __restrict__ c,
                                const double* __restrict__ kk) {
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < lines;
         L += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = L / (ny * nz);
        thomas(rho + L * nx, 1, nx, kk[s], m + (size_t)(3 * s) * nmax, c + (size_t)(3 * s) * nmax);
    }
}

// y lines (axis 1) or z lines (axis 2): thread t = (s, outer, x); consecutive
// threads are consecutive x, so every step of the recurrence is coalesced.
__global__ void k_diff_yz(double* __restrict__ rho, int axis, int32_t S, int64_t nx, int64_t ny, int64_t nz,
                          int64_t nmax, const double* __restrict__ m, const double* __restrict__ c,
                          const double* __restrict__ kk) {
    const int64_t nv = nx * ny * nz;
    const int64_t outer = axis == 1 ? nz : ny;
    const int64_t lines = (int64_t)S * outer * nx;
    const int64_t n = axis == 1 ? ny : nz;
    const int64_t stride = axis == 1 ? nx : nx * ny;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < lines; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = t % nx;
        const int64_t r = t / nx;
        const int64_t o = r % outer;
        const int64_t s = r / outer;
        const int64_t base = s * nv + x + (axis == 1 ? o * nx * ny : o * nx);
        thomas(rho + base, stride, n, kk[s], m + (size_t)(3 * s + axis) * nmax, c + (size_t)(3 * s + axis) * nmax);
    }
}

__global__ void k_diff_gradient(const double* __restrict__ rho, int32_t S, int64_t nx, int64_t ny, int64_t nz,
                                double dx, double* __restrict__ grad) {
    const int64_t nv = nx * ny * nz;
    const int64_t total = (int64_t)S * nv;
    const double two_dx = __dmul_rn(2.0, dx);
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = t / nv, v = t - s * nv;
        const int64_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
        const double* r = rho + s * nv;
        const int64_t n[3] = {nx, ny, nz};
        const int64_t i[3] = {x, y, z};
        const int64_t st[3] = {1, nx, nx * ny};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double g;
            if (n[a] == 1) g = 0.0;
            else if (i[a] == 0) g = __ddiv_rn(__dsub_rn(r[v + st[a]], r[v]), dx);
            else if (i[a] == n[a] - 1) g = __ddiv_rn(__dsub_rn(r[v], r[v - st[a]]), dx);
            else g = __ddiv_rn(__dsub_rn(r[v + st[a]], r[v - st[a]]), two_dx);
            grad[(s * 3 + a) * nv + v] = g;
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
    if (rc == MECH_OK) rc = h->alloc(&h->d_k, (size_t)h->S);
    if (rc != MECH_OK) return bail(rc);
    rc = dcuda(cudaMemcpyAsync(h->d_D, D, h->S * 8, cudaMemcpyHostToDevice, h->stream), "upload D");
    if (rc == MECH_OK) rc = dcuda(cudaMemcpyAsync(h->d_lam, lambda, h->S * 8, cudaMemcpyHostToDevice, h->stream),
                                  "upload lambda");
    if (rc == MECH_OK) rc = dcuda(cudaMemsetAsync(h->d_rho, 0, nvals * 8, h->stream), "zero densities");
    if (rc == MECH_OK) rc = dcuda(cudaStreamSynchronize(h->stream), "create");
    if (rc != MECH_OK) return bail(rc);
    // the staged x tile needs at most 32 x 191 doubles = 48,896 bytes, within
    // the default 48 KiB of dynamic shared memory: no per-function attribute
    // (a process-wide setting) is changed
    static_assert(kLineTile * kMaxNxTile * sizeof(double) <= 48 * 1024, "x tile within the default limit");
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
                                                                               h->d_c, h->d_k);
        DTRY(dcuda(cudaGetLastError(), "coefficients"));
        h->dt_coef = dt;
    }
    const int64_t xlines = (int64_t)h->S * h->ny * h->nz;
    const int64_t ylines = (int64_t)h->S * h->nz * h->nx;
    const int64_t zlines = (int64_t)h->S * h->ny * h->nx;
    const int xblocks = grid_for(xlines, kLineTile, h->sms);
    const int xbytes = (int)(kLineTile * (h->nx | 1) * sizeof(double));
    for (int64_t step = 0; step < n_steps; ++step) {
        if (h->nx <= kMaxNxTile)
            k_diff_x_tiled<<<xblocks, kLineTile, xbytes, h->stream>>>(h->d_rho, xlines, h->nx, h->ny, h->nz, h->nmax,
                                                                      h->d_m, h->d_c, h->d_k);
        else
            k_diff_x_direct<<<grid_for(xlines, 128, h->sms), 128, 0, h->stream>>>(h->d_rho, xlines, h->nx, h->ny,
                                                                                  h->nz, h->nmax, h->d_m, h->d_c,
                                                                                  h->d_k);
        k_diff_yz<<<grid_for(ylines, 128, h->sms), 128, 0, h->stream>>>(h->d_rho, 1, h->S, h->nx, h->ny, h->nz,
                                                                        h->nmax, h->d_m, h->d_c, h->d_k);
        k_diff_yz<<<grid_for(zlines, 128, h->sms), 128, 0, h->stream>>>(h->d_rho, 2, h->S, h->nx, h->ny, h->nz,
                                                                        h->nmax, h->d_m, h->d_c, h->d_k);
        DTRY(dcuda(cudaGetLastError(), "diffusion step"));
    }
    return MECH_OK;
}

int mech_diffusion_gradient(mech_diffusion_t* h, double* grad) {
    DTRY(dcheck(h));
    k_diff_gradient<<<grid_for((int64_t)h->S * h->nv, 256, h->sms), 256, 0, h->stream>>>(h->d_rho, h->S, h->nx, h->ny,
                                                                                        h->nz, h->dx, h->d_grad);
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
