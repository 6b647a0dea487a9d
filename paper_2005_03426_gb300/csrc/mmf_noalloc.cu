// mmf_noalloc.cu -- the tridiagonal eigensolver (bisection + inverse iteration) for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host program whose device memory is entirely owned by
// another allocator (for example a framework's caching allocator that has already reserved the
// HBM), or a latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation.  For them this entry point runs the same tridiagonal eigensolver kernels as
// the batched path, with every scratch buffer carved from one file-scope device array of fixed
// size instead of allocated memory.  The caller passes the inputs (d, e) and outputs (E, Y) as
// device pointers.
//
// The scratch array below occupies MMF_NOALLOC_SCRATCH_BYTES (about 1.6 MB) on every GPU that
// loads the library, until the process exits.  All calls share it: the status word is cleared
// at the start of each call, everything else is written before it is read, and calls whose GPU
// work overlaps (on different streams, or from several host threads) race on it.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <string>

#include "../../include/mmf.h"
#include "mmf_internal.h"

int mmf_set_error(int code, const std::string& msg);

// Layout of the scratch (bytes): descriptor | index + status | aux (8 doubles) | e^2 (NMAX
// doubles) | inverse-iteration factors (3 NMAX^2 doubles).
#define NA_OFF_DESC 0
#define NA_OFF_INT 256
#define NA_OFF_AUX 512
#define NA_OFF_E2 (NA_OFF_AUX + 8 * 8)
#define NA_OFF_WORK (((NA_OFF_E2 + 8 * MMF_NOALLOC_TRIDIAG_NMAX) + 255) / 256 * 256)
#define MMF_NOALLOC_SCRATCH_BYTES \
    (NA_OFF_WORK + 8 * 3 * MMF_NOALLOC_TRIDIAG_NMAX * MMF_NOALLOC_TRIDIAG_NMAX)

static_assert(sizeof(MmfDesc) <= NA_OFF_INT, "descriptor slot too small");

static __device__ __align__(256) unsigned char g_tridiag_scratch[MMF_NOALLOC_SCRATCH_BYTES];

// Device addresses of the scratch array, looked up once per device (the symbol's host-side
// name is only a stand-in for it and must never be handed to a kernel).
#define NA_MAX_DEVICES 64
static unsigned char* g_scratch_addr[NA_MAX_DEVICES];
static std::mutex g_scratch_mu;

static int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mmf_set_error(MMF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return mmf_set_error(MMF_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tridiag_scratch);
        if (e != cudaSuccess || !p)
            return mmf_set_error(MMF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_scratch_addr[dev] = (unsigned char*)p;
    }
    *out = g_scratch_addr[dev];
    return MMF_OK;
}

extern "C" int mmf_tridiag_eig_noalloc(const double* d, const double* e, int n, double* E, double* Y,
                                       void* stream) {
    if (n < 1 || n > MMF_NOALLOC_TRIDIAG_NMAX)
        return mmf_set_error(MMF_ERR_UNSUPPORTED,
                             "mmf_tridiag_eig_noalloc: n = " + std::to_string(n) + " outside 1.." +
                                 std::to_string(MMF_NOALLOC_TRIDIAG_NMAX) + " (fixed scratch size)");
    if (!d || !E || !Y || (n > 1 && !e)) return mmf_set_error(MMF_ERR_ARG, "d, e, E and Y are required");
    unsigned char* s = nullptr;
    int rc = scratch_for_current_device(&s);
    if (rc != MMF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    MmfDesc desc;
    std::memset(&desc, 0, sizeof(desc));
    desc.n = n;
    desc.D = 1;
    desc.M = n;
    desc.ld = n;
    const int idx0 = 0;
    cudaError_t err = cudaMemcpyAsync(s + NA_OFF_DESC, &desc, sizeof(desc), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemcpyAsync(s + NA_OFF_INT, &idx0, sizeof(int), cudaMemcpyHostToDevice, st);
    if (err == cudaSuccess) err = cudaMemsetAsync(s + NA_OFF_INT + sizeof(int), 0, sizeof(int), st);
    if (err != cudaSuccess)
        return mmf_set_error(MMF_ERR_CUDA, std::string("mmf_tridiag_eig_noalloc set-up: ") + cudaGetErrorString(err));
    MmfLaunch L;
    L.desc = (const MmfDesc*)(s + NA_OFF_DESC);
    L.idx = (const int*)(s + NA_OFF_INT);
    L.count = 1;
    L.nmax = n;
    L.stream = st;
    err = mmf_launch_tridiag_eig(L, d, e, (double*)(s + NA_OFF_AUX), (double*)(s + NA_OFF_E2), E, Y,
                                 (double*)(s + NA_OFF_WORK), (int*)(s + NA_OFF_INT + sizeof(int)),
                                 0, 3);
    if (err != cudaSuccess)
        return mmf_set_error(MMF_ERR_CUDA, std::string("mmf_tridiag_eig_noalloc: ") + cudaGetErrorString(err));
    return MMF_OK;
}
