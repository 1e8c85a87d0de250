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

// Driver-API entry points, fetched through the runtime (no link against
// libcuda): the current context and its process-unique ID.
typedef int (*CtxGetCurrentFn)(void **ctx);
typedef int (*CtxGetIdFn)(void *ctx, unsigned long long *id);

std::mutex g_lock;
bool g_fns_tried = false;
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;

// Device address of g_dt_partial per device ordinal, with the ID of the context
// it was looked up in.  A context made again after cudaDeviceReset (or after the
// primary context was released) has another ID, and the address is looked up
// again, because the module, and with it the array, may then sit elsewhere.
struct SymbolSlot {
    unsigned long long ctx_id;
    double *addr;
};
SymbolSlot g_slot[256];

// ID of the calling thread's current context (0 when it has none or the driver
// cannot say).
unsigned long long current_ctx_id()
{
    if (!g_fns_tried) {
        g_fns_tried = true;
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = (CtxGetCurrentFn)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = (CtxGetIdFn)f;
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx) return 0;
    if (g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

}  // namespace

extern "C" pd_status pd_stable_dt_noalloc(int64_t n, const double *x, const double *vol, const int64_t *rowptr,
                                          const int32_t *col, double c, double rho, void *stream, double *dt_out)
{
    if (n < 1 || !x || !vol || !rowptr || !col || !dt_out || !(c > 0) || !(rho > 0)) return PD_EINVAL;
    if (n > (int64_t)PD_NOALLOC_MAX_BLOCKS * PD_NOALLOC_ROWS_PER_BLOCK) return PD_EINVAL;  // scratch too small
    // an error some earlier call left pending is the caller's: it is neither
    // reported as this call's failure nor cleared by it
    const bool pending = cudaPeekAtLastError() != cudaSuccess;
    auto failed = [&]() {
        if (!pending) cudaGetLastError();  // clear only what this call raised
        return PD_ECUDA;
    };
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return failed();
    double *partial;
    {
        std::lock_guard<std::mutex> guard(g_lock);
        unsigned long long id = current_ctx_id();
        SymbolSlot &slot = g_slot[dev];
        if (!slot.addr || id == 0 || id != slot.ctx_id) {
            // host code cannot use the array's name as a device address: ask the
            // runtime for this device's copy (first call on a device, first call in
            // a new context, or every call where the context ID is unknown).  This
            // also makes the runtime create the primary context if there is none.
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_dt_partial) != cudaSuccess || !ptr) return failed();
            if (id == 0) id = current_ctx_id();
            slot.addr = (double *)ptr;
            slot.ctx_id = id;
        }
        partial = slot.addr;
    }
    const int nb = (int)((n + PD_NOALLOC_ROWS_PER_BLOCK - 1) / PD_NOALLOC_ROWS_PER_BLOCK);
    cudaStream_t st = (cudaStream_t)stream;
    // launch status from the launch calls themselves, not from the thread's last
    // error (which may hold the caller's)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nb);
    cfg.blockDim = dim3(PD_NOALLOC_ROWS_PER_BLOCK);
    cfg.stream = st;
    if (cudaLaunchKernelEx(&cfg, k_dt_partial, x, vol, rowptr, col, n, c, rho, partial) != cudaSuccess)
        return failed();
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(256);
    if (cudaLaunchKernelEx(&cfg, k_dt_final, (const double *)partial, nb, dt_out) != cudaSuccess) return failed();
    return PD_OK;
}
