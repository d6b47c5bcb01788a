// Allocation-free variant of the FP64 block solve (gwas_solve_block_noalloc).
//
// Some callers cannot allocate device memory when they call into this library: their
// GPU memory is already fully reserved by another allocator (a framework's caching
// allocator, or a fixed memory budget per process), or they run a latency-sensitive
// serving loop in which cudaMalloc/cudaFree, which may synchronise the device, are not
// acceptable. For them this entry point runs the same two kernels as the FP64 block
// path (k_block_fp64, k_snp_solve) on buffers the caller passes in, and takes the
// kernels' scratch (row-tile partial sums and per-SNP dosage flags) from one
// fixed-size array in device global memory that is part of the library image itself.
// The array exists on every GPU that loads the library, from load until process exit.
#include <mutex>

#include "../../include/gwas.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB

// Scratch of gwas_solve_block_noalloc. In host code this name is only a host-side
// stand-in for the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_dev[kMaxDevices] = {};  // device address of the array, per device

// Device address of the scratch array on the current device, looked up once per device.
gwas_status scratch_on_current_device(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return GWAS_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevices) return GWAS_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return GWAS_ERR_CUDA;
        }
        g_scratch_dev[dev] = p;
    }
    *out = g_scratch_dev[dev];
    return GWAS_OK;
}

// True when bytes [p, p + bytes) start and end in device (or managed) memory of device
// `dev`. Allocates nothing; an address the runtime does not know (host memory, a
// foreign device's pointer, a stray integer) is refused before any kernel sees it.
bool device_range(const void* p, size_t bytes, int dev) {
    if (!p || bytes == 0) return false;
    const unsigned char* ends[2] = {static_cast<const unsigned char*>(p),
                                    static_cast<const unsigned char*>(p) + (bytes - 1)};
    for (const unsigned char* q : ends) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged) return false;
        if (at.device != dev) return false;
    }
    return true;
}

}  // namespace

extern "C" gwas_status gwas_solve_block_noalloc(int64_t n, int p, int t, const double* Linv,
                                                int64_t ld_linv, const double* XLbar,
                                                const double* Ybar, const double* S_TL,
                                                const double* bbar_T, const int8_t* X,
                                                int64_t mb, double* b, double* wald,
                                                uint8_t* status, void* stream) {
    using namespace gwas;
    if (n < 1 || p < 2 || p > MAX_P || t < 1 || t > MAX_T || mb < 1 || ld_linv < n)
        return GWAS_ERR_ARG;
    if (!Linv || !XLbar || !Ybar || !S_TL || !bbar_T || !X || !b || !status) return GWAS_ERR_ARG;
    const int64_t n_rt = ceil_div(n, T64);
    const int64_t ldp = round_up(mb, 32);
    const int64_t nred = (int64_t)p + t;  // (p-1) + 1 + t reduction values per SNP
    const int64_t part_bytes = round_up(n_rt * nred * ldp * (int64_t)sizeof(double), 256);
    const int64_t bad_bytes = round_up(mb, 256);
    if (part_bytes + bad_bytes > (int64_t)kScratchBytes) return GWAS_ERR_TOO_LARGE;

    // every buffer must be device memory of the current device, large enough for the call
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return GWAS_ERR_CUDA;
    }
    const size_t d8 = sizeof(double);
    const int64_t q = p - 1;
    if (!device_range(Linv, (size_t)(ld_linv * (n - 1) + n) * d8, dev) ||
        !device_range(XLbar, (size_t)(n * q) * d8, dev) ||
        !device_range(Ybar, (size_t)(n * t) * d8, dev) ||
        !device_range(S_TL, (size_t)(q * q) * d8, dev) ||
        !device_range(bbar_T, (size_t)(q * t) * d8, dev) ||
        !device_range(X, (size_t)(n * mb), dev) ||
        !device_range(b, (size_t)(mb * t * p) * d8, dev) ||
        (wald && !device_range(wald, (size_t)(mb * t) * d8, dev)) ||
        !device_range(status, (size_t)mb, dev))
        return GWAS_ERR_ARG;

    void* base = nullptr;
    const gwas_status st = scratch_on_current_device(&base);
    if (st != GWAS_OK) return st;
    double* part = static_cast<double*>(base);
    uint8_t* bad = static_cast<uint8_t*>(base) + part_bytes;

    CohortDev c;
    c.n = n; c.q = p - 1; c.t = t;
    c.W = Linv; c.ldw = ld_linv;
    c.XLbar = XLbar; c.Ybar = Ybar; c.S_TL = S_TL; c.bbar_T = bbar_T;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Every partial and flag the solve reads is written by k_block_fp64 first, so the
    // previous call's contents never need clearing.
    if (launch_block_fp64(c, X, n, mb, part, ldp, bad, s) != cudaSuccess) return GWAS_ERR_CUDA;
    if (launch_snp_solve(c, part, ldp, (int)n_rt, bad, mb, b, wald, status, s) != cudaSuccess)
        return GWAS_ERR_CUDA;
    return GWAS_OK;
}
