// Allocation-free variant of the critical-time-step reduction.
//
// pd_stable_dt (pd_api.cu) keeps its per-block partial minima in memory the
// context allocated.  Some callers cannot allocate device memory at the moment
// they need the step: code running while a memory pool is frozen, an embedding
// runtime that owns every device allocation itself, or a host callback where
// cudaMalloc is not allowed.  pd_stable_dt_noalloc takes the caller's device
// arrays and writes the result to the caller's device double; its only scratch
// is the file-scope array below, which exists once per GPU that loads this
// library and lives until the process exits.
#include <mutex>

#include "pd_internal.cuh"

#define PD_NOALLOC_ROWS_PER_BLOCK 256
#define PD_NOALLOC_MAX_BLOCKS 65536  // 512 KiB of partials: n <= 16,777,216 nodes

static __device__ __align__(256) double g_dt_partial[PD_NOALLOC_MAX_BLOCKS];

namespace {

// one block per 256 rows: min over its rows of sqrt(2 rho / sum_j V_j c / |xi_ij|)
__global__ void k_dt_partial(const double *__restrict__ x, const double *__restrict__ vol,
                             const int64_t *__restrict__ rowptr, const int32_t *__restrict__ col, int64_t n,
                             double c, double rho, double *partial)
{
    __shared__ double s_min[PD_NOALLOC_ROWS_PER_BLOCK];
    const int64_t i = (int64_t)blockIdx.x * PD_NOALLOC_ROWS_PER_BLOCK + threadIdx.x;
    double best = INFINITY;
    if (i < n) {
        const int64_t k0 = rowptr[i], k1 = rowptr[i + 1];
        if (k1 > k0) {
            const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
            double sum = 0.0;
            for (int64_t k = k0; k < k1; ++k) {
                const int64_t j = col[k];
                const double dx = x[3 * j] - xi, dy = x[3 * j + 1] - yi, dz = x[3 * j + 2] - zi;
                sum += vol[j] * c / sqrt(dx * dx + dy * dy + dz * dz);
            }
            best = sqrt(2.0 * rho / sum);
        }
    }
    s_min[threadIdx.x] = best;
    __syncthreads();
    for (int o = PD_NOALLOC_ROWS_PER_BLOCK / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = s_min[0];
}

__global__ void k_dt_final(const double *__restrict__ partial, int nb, double *out)
{
    __shared__ double s_min[256];
    double m = INFINITY;
    for (int b = threadIdx.x; b < nb; b += 256) m = fmin(m, partial[b]);
    s_min[threadIdx.x] = m;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) s_min[threadIdx.x] = fmin(s_min[threadIdx.x], s_min[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = s_min[0];
}

std::mutex g_lock;
double *g_addr[256];  // device address of g_dt_partial, per device ordinal (set up once)

}  // namespace

extern "C" pd_status pd_stable_dt_noalloc(int64_t n, const double *x, const double *vol, const int64_t *rowptr,
                                          const int32_t *col, double c, double rho, void *stream, double *dt_out)
{
    if (n < 1 || !x || !vol || !rowptr || !col || !dt_out || !(c > 0) || !(rho > 0)) return PD_EINVAL;
    if (n > (int64_t)PD_NOALLOC_MAX_BLOCKS * PD_NOALLOC_ROWS_PER_BLOCK) return PD_EINVAL;  // scratch too small
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) {
        cudaGetLastError();
        return PD_ECUDA;
    }
    double *partial;
    {
        std::lock_guard<std::mutex> guard(g_lock);
        if (!g_addr[dev]) {
            // host code cannot use the array's name as a device address: ask the
            // runtime for this device's copy (first call on each device)
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_dt_partial) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PD_ECUDA;
            }
            g_addr[dev] = (double *)ptr;
        }
        partial = g_addr[dev];
    }
    const int nb = (int)((n + PD_NOALLOC_ROWS_PER_BLOCK - 1) / PD_NOALLOC_ROWS_PER_BLOCK);
    cudaStream_t st = (cudaStream_t)stream;
    k_dt_partial<<<nb, PD_NOALLOC_ROWS_PER_BLOCK, 0, st>>>(x, vol, rowptr, col, n, c, rho, partial);
    k_dt_final<<<1, 256, 0, st>>>(partial, nb, dt_out);
    if (cudaGetLastError() != cudaSuccess) return PD_ECUDA;
    return PD_OK;
}
