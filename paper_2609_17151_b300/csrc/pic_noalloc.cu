// pic_noalloc.cu -- counting sort by cell that allocates no device memory.
//
// pic_sort_by_cell takes its per-call scratch (per-cell counts and cursors)
// from the stream-ordered allocator.  Some callers must not allocate device
// memory once they are running: an application that fixes its device-memory
// budget at start-up, a plug-in inside a host program that owns the whole
// device heap through its own allocator, or a loop that cannot afford the
// device-wide synchronisation that cudaMalloc / cudaFree can imply.  For them,
// pic_sort_by_cell_noalloc does the same sort with its scratch in one fixed,
// library-owned device array declared below (sized for PIC_NOALLOC_MAX_CELLS
// cells; every device that loads this library keeps it until the process
// exits).  The caller still provides the input and output particle arrays.
#include "pic1d3v.h"

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

namespace pic {
void set_last_error(const std::string &msg);      // defined with pic_last_error
}

namespace {

constexpr int kMaxCells = PIC_NOALLOC_MAX_CELLS;
constexpr int kChunk = 8192;                     // particles per CTA in the scatter
constexpr int kMaxDevices = 64;

// Scratch layout (64-bit words): counts, kMaxCells x uint32 (= kMaxCells/2
// words), then cursors, (kMaxCells + 1) x uint64.  49,160 bytes.
constexpr int kCountWords = kMaxCells / 2;
constexpr int kScratchWords = kCountWords + kMaxCells + 1;
static __device__ __align__(256) unsigned long long g_sort_scratch[kScratchWords];

// Device address of g_sort_scratch per device.  In host code the symbol's
// name is only a host-side stand-in; the address comes from
// cudaGetSymbolAddress with the device current.
std::mutex g_setup_mutex;
unsigned long long *g_scratch_ptr[kMaxDevices] = {};

struct Soa {
    const int32_t *cell;
    const float *off, *vx, *vy, *vz;
    const uint32_t *id;
};
struct SoaOut {
    int32_t *cell;
    float *off, *vx, *vy, *vz;
    uint32_t *id;
};

__global__ void k_na_count(Soa A, long long n, int N, unsigned *counts)
{
    extern __shared__ unsigned cnt_s[];
    for (int j = threadIdx.x; j < N; j += blockDim.x) cnt_s[j] = 0u;
    __syncthreads();
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int c = A.cell[i];
        if (c >= 0 && c < N) atomicAdd(&cnt_s[c], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x)
        if (cnt_s[j]) atomicAdd(&counts[j], cnt_s[j]);
}

// One CTA: cursor[j] = sum_{k<j} counts[k], cursor[N] = total (64-bit, exact).
__global__ void __launch_bounds__(1024) k_na_scan(const unsigned *counts, int N, unsigned long long *cursor)
{
    __shared__ unsigned long long warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const int per = (N + blockDim.x - 1) / blockDim.x;
    const int lo = min(tid * per, N), hi = min(lo + per, N);
    unsigned long long s = 0;
    for (int j = lo; j < hi; ++j) s += counts[j];
    unsigned long long incl = s;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    unsigned long long off = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        if (w < warp) off += warp_tot[w];
        tot += warp_tot[w];
    }
    unsigned long long run = off + incl - s;
    for (int j = lo; j < hi; ++j) {
        cursor[j] = run;
        run += counts[j];
    }
    if (tid == 0) cursor[N] = tot;
}

__global__ void k_na_scatter(Soa A, SoaOut D, long long n, int N, unsigned long long *cursor)
{
    extern __shared__ __align__(16) unsigned char xsm[];
    unsigned long long *base = reinterpret_cast<unsigned long long *>(xsm);
    unsigned *lcnt = reinterpret_cast<unsigned *>(xsm + 8 * (size_t)N);
    for (int j = threadIdx.x; j < N; j += blockDim.x) lcnt[j] = 0u;
    __syncthreads();
    const long long lo = (long long)blockIdx.x * kChunk, hi = min(lo + kChunk, n);
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int c = A.cell[i];
        if (c >= 0 && c < N) atomicAdd(&lcnt[c], 1u);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const unsigned k = lcnt[j];
        base[j] = k ? atomicAdd(&cursor[j], (unsigned long long)k) : 0ull;
        lcnt[j] = 0u;
    }
    __syncthreads();
    for (long long i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const int c = A.cell[i];
        if (c < 0 || c >= N) continue;
        const unsigned long long p = base[c] + atomicAdd(&lcnt[c], 1u);
        D.cell[p] = c; D.off[p] = A.off[i]; D.vx[p] = A.vx[i]; D.vy[p] = A.vy[i]; D.vz[p] = A.vz[i];
        D.id[p] = A.id[i];
    }
}

pic_status na_fail(pic_status s, const std::string &msg)
{
    pic::set_last_error(msg);             // reported by pic_last_error()
    return s;
}

// The device address of the scratch array for the current device, looked up
// once per device (the first call on a device does this).
pic_status scratch_for_current_device(unsigned long long **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return na_fail(PIC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return na_fail(PIC_EINVAL, "device ordinal beyond the supported range");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        unsigned long long *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_sort_scratch);
        if (e != cudaSuccess || !p)
            return na_fail(PIC_ECUDA, std::string("cudaGetSymbolAddress(scratch): ") + cudaGetErrorString(e));
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return PIC_OK;
}

} // namespace

extern "C" {

pic_status pic_sort_by_cell_noalloc(int32_t n_cells, int64_t n, const int32_t *cell, const float *off,
                                    const float *vx, const float *vy, const float *vz, const uint32_t *id,
                                    int32_t *cell_out, float *off_out, float *vx_out, float *vy_out,
                                    float *vz_out, uint32_t *id_out, int64_t *n_live, void *stream)
{
    if (n_cells < 1 || n_cells > kMaxCells)
        return na_fail(PIC_EINVAL, "n_cells must be in [1, PIC_NOALLOC_MAX_CELLS = " + std::to_string(kMaxCells) +
                                       "] for the allocation-free sort");
    if (n < 0) return na_fail(PIC_EINVAL, "n must be >= 0");
    if (n > 0 && (!cell || !off || !vx || !vy || !vz || !id || !cell_out || !off_out || !vx_out || !vy_out ||
                  !vz_out || !id_out))
        return na_fail(PIC_EINVAL, "null particle array");
    unsigned long long *scratch = nullptr;
    pic_status st = scratch_for_current_device(&scratch);
    if (st != PIC_OK) return st;
    unsigned *counts = reinterpret_cast<unsigned *>(scratch);
    unsigned long long *cursor = scratch + kCountWords;
    cudaStream_t s = (cudaStream_t)stream;
    const int N = n_cells;
    // the array keeps the previous call's contents: clear what must start at zero
    cudaError_t e = cudaMemsetAsync(counts, 0, (size_t)N * sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor + N, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return na_fail(PIC_ECUDA, std::string("scratch clear: ") + cudaGetErrorString(e));
    if (n > 0) {
        int dev = 0, sms = 148;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const Soa A{cell, off, vx, vy, vz, id};
        const SoaOut D{cell_out, off_out, vx_out, vy_out, vz_out, id_out};
        const long long gc = n / 1024 < 1 ? 1 : (n / 1024 < 4LL * sms ? n / 1024 : 4LL * sms);
        k_na_count<<<(unsigned)gc, 512, N * sizeof(unsigned), s>>>(A, n, N, counts);
        k_na_scan<<<1, 1024, 0, s>>>(counts, N, cursor);
        k_na_scatter<<<(unsigned)((n + kChunk - 1) / kChunk), 512, 12 * (size_t)N, s>>>(A, D, n, N, cursor);
        e = cudaGetLastError();
        if (e != cudaSuccess) return na_fail(PIC_ECUDA, std::string("sort launch: ") + cudaGetErrorString(e));
    }
    if (n_live) {
        e = cudaMemcpyAsync(n_live, cursor + N, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return na_fail(PIC_ECUDA, std::string("count copy: ") + cudaGetErrorString(e));
    }
    return PIC_OK;
}

} // extern "C"
