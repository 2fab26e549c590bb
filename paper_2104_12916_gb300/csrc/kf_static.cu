// kf_static.cu -- qp_kf_apply_static: the implicit K_F product with no device
// allocation (declared in include/pcgipm.h).
//
// For callers that cannot allocate device memory themselves (code that runs
// under an allocator it does not own, inside a region where cudaMalloc would
// synchronise the device or is forbidden, or on a memory budget fixed in
// advance).  The caller passes every input and the output; the intermediate
// vectors live in the file-scope array below.  Under CUDA's lazy module loading
// (the default since CUDA 12.2) the array is reserved in a device's memory when
// this module is first used on that device -- at the first cudaGetSymbolAddress
// or launch -- and kept until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/pcgipm.h"

namespace {

// Intermediate vectors u, z1, t, y (n each) and z2 (m1): 4 n + m1 doubles.
constexpr int kStaticMaxN = QP_STATIC_MAX_N;
constexpr size_t kStaticDoubles = 4 * (size_t)kStaticMaxN + (size_t)kStaticMaxN;

static __device__ __align__(256) double g_kf_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_kf_scratch for the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_kf_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Row product over a row-major matrix (leading dimension = cols), one warp per
// row, columns [lo(i), hi(i)): lower == 1 restricts row i to columns [0, i].
// y_i = a * (M x)_i + b * z_i + dv_i * px_i  (z, dv may be null).
__global__ void row_gemv(const double* __restrict__ M, int rows, int cols, int lower,
                         const double* __restrict__ x, double a, const double* __restrict__ z, double b,
                         const double* __restrict__ dv, const double* __restrict__ px, double* __restrict__ y) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= rows) return;
    const int hi = lower ? min(cols, warp + 1) : cols;
    const double* mr = M + (long long)warp * cols;
    double s = 0.0;
    for (int j = lane; j < hi; j += 32) s = fma(mr[j], x[j], s);
    s = warp_sum(s);
    if (lane == 0) {
        double v = a * s;
        if (z) v += b * z[warp];
        if (dv) v += dv[warp] * px[warp];
        y[warp] = v;
    }
}

// Column product over a row-major matrix: y_j = a * sum_i M_ij x_i + b * z_j,
// one thread per column (coalesced across threads); lower == 1 restricts column
// j to rows [j, rows).
__global__ void col_gemv(const double* __restrict__ M, int rows, int cols, int lower,
                         const double* __restrict__ x, double a, const double* __restrict__ z, double b,
                         double* __restrict__ y) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= cols) return;
    double s = 0.0;
    for (int i = lower ? j : 0; i < rows; ++i) s = fma(M[(long long)i * cols + j], x[i], s);
    double v = a * s;
    if (z) v += b * z[j];
    y[j] = v;
}

}  // namespace

extern "C" int qp_kf_apply_static(int n, int m1, int m2, const double* C, const double* WH, const double* Gt,
                                  const double* D, const double* p, double* q, void* stream) {
    if (n < 1 || n > kStaticMaxN || m1 < 0 || m1 > n || m2 < 1) return QP_EINVAL;
    if (!C || !WH || !D || !p || !q || (m1 > 0 && !Gt)) return QP_EINVAL;
    // An error left pending by an earlier, unrelated call is reported (and left in
    // place for its owner) instead of being mistaken for one of this call's launches.
    if (cudaPeekAtLastError() != cudaSuccess) return QP_ECUDA;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return QP_ECUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* u = scratch;
    double* z1 = u + kStaticMaxN;
    double* t = z1 + kStaticMaxN;
    double* y = t + kStaticMaxN;
    double* z2 = y + kStaticMaxN;
    const int T = 256;
    auto rows_grid = [&](int rows) { return (rows * 32 + T - 1) / T; };
    auto cols_grid = [&](int cols) { return (cols + T - 1) / T; };
    // u = C' p
    col_gemv<<<cols_grid(n), T, 0, s>>>(C, m2, n, 0, p, 1.0, nullptr, 0.0, u);
    // z1 = R^{-T} u  (WH lower)
    row_gemv<<<rows_grid(n), T, 0, s>>>(WH, n, n, 1, u, 1.0, nullptr, 0.0, nullptr, nullptr, z1);
    const double* top = z1;
    if (m1 > 0) {
        // z2 = -Gt z1 ;  t = z1 + Gt' z2
        row_gemv<<<rows_grid(m1), T, 0, s>>>(Gt, m1, n, 0, z1, -1.0, nullptr, 0.0, nullptr, nullptr, z2);
        col_gemv<<<cols_grid(n), T, 0, s>>>(Gt, m1, n, 0, z2, 1.0, z1, 1.0, t);
        top = t;
    }
    // y = R^{-1} top = WH' top  (column product over the lower triangle)
    col_gemv<<<cols_grid(n), T, 0, s>>>(WH, n, n, 1, top, 1.0, nullptr, 0.0, y);
    // q = D p + C y
    row_gemv<<<rows_grid(m2), T, 0, s>>>(C, m2, n, 0, y, 1.0, nullptr, 0.0, D, p, q);
    // launch errors only: an error during execution shows at the caller's next
    // synchronisation with the stream
    if (cudaGetLastError() != cudaSuccess) return QP_ECUDA;
    return QP_OK;
}
