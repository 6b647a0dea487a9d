// mmf_noalloc.cu -- the tridiagonal eigensolver (bisection + inverse iteration) for callers
// that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: a host program whose device memory is entirely owned by
// another allocator (for example a framework's caching allocator that has already reserved the
// HBM), or a latency-critical loop that cannot afford cudaMalloc's implicit device
// synchronisation.  For them this entry point runs the same tridiagonal eigensolver kernels as
// the batched path, with every scratch buffer carved from one file-scope device array of fixed
// size instead of allocated memory.  The caller passes the inputs (d, e) and outputs (E, Y, and
// optionally a status word) as device pointers.
//
// The scratch array below occupies MMF_NOALLOC_SCRATCH_BYTES (about 1.6 MB) on every GPU that
// loads the library, until the process exits.  All calls share it.  Each call first enqueues a
// one-thread set-up kernel that writes the solver's descriptor and system index into the array
// and clears the status word (kernel arguments only: no host copy, so the call never waits for
// the stream); everything else in the array is written before it is read.  Calls whose GPU work
// overlaps (on different streams, or from several host threads) race on the array.
#include <cuda.h>
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
static_assert(sizeof(MmfDesc) % sizeof(int) == 0, "descriptor is written as whole ints");

static __device__ __align__(256) unsigned char g_tridiag_scratch[MMF_NOALLOC_SCRATCH_BYTES];

// Writes the descriptor of one n x n tridiagonal system (all offsets 0), its index and a cleared
// status word into the scratch array.
__global__ void k_noalloc_setup(MmfDesc* desc, int* idx, int* status, int n) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int* w = reinterpret_cast<int*>(desc);
    for (int i = 0; i < (int)(sizeof(MmfDesc) / sizeof(int)); ++i) w[i] = 0;
    desc->n = n;
    desc->D = 1;
    desc->M = n;
    desc->ld = n;
    idx[0] = 0;
    *status = MMF_ST_OK;
}

// Device address of the scratch array in the current context.  The symbol's host-side name is
// only a stand-in for it and must never be handed to a kernel.  The address is looked up once per
// device and context: a context is recognised by the driver's unique context id (cuCtxGetId,
// reached through the runtime's driver entry points, so the library need not link libcuda), so
// the lookup is repeated after the context was reset.  If those entry points are unavailable the
// address is looked up on every call.
typedef CUresult (*PfnCtxGetCurrent)(CUcontext*);
typedef CUresult (*PfnCtxGetId)(CUcontext, unsigned long long*);

#define NA_MAX_DEVICES 64
struct ScratchCache {
    unsigned long long ctx_id = 0;
    unsigned char* addr = nullptr;
};
static ScratchCache g_cache[NA_MAX_DEVICES];
static std::mutex g_scratch_mu;
static PfnCtxGetCurrent g_get_current = nullptr;
static PfnCtxGetId g_get_id = nullptr;
static bool g_entry_points_tried = false;

static bool current_context_id(unsigned long long* id) {
    if (!g_entry_points_tried) {
        g_entry_points_tried = true;
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) ==
                cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess && f1 && f2) {
            g_get_current = (PfnCtxGetCurrent)f1;
            g_get_id = (PfnCtxGetId)f2;
        }
    }
    if (!g_get_current || !g_get_id) return false;
    CUcontext ctx = nullptr;
    if (g_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_get_id(ctx, id) == CUDA_SUCCESS;
}

static int scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return mmf_set_error(MMF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= NA_MAX_DEVICES) return mmf_set_error(MMF_ERR_UNSUPPORTED, "device index above 63");
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    ScratchCache& c = g_cache[dev];
    if (!have_id || !c.addr || c.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_tridiag_scratch);
        if (e != cudaSuccess || !p)
            return mmf_set_error(MMF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        // the lookup may have created the context: take its id now
        unsigned long long id2 = 0;
        const bool have_id2 = current_context_id(&id2);
        c.addr = (unsigned char*)p;
        c.ctx_id = have_id2 ? id2 : 0;
        if (!have_id2) {  // no context id: do not keep the address
            *out = c.addr;
            c.addr = nullptr;
            return MMF_OK;
        }
    }
    *out = c.addr;
    return MMF_OK;
}

extern "C" int mmf_tridiag_eig_noalloc(const double* d, const double* e, int n, double* E, double* Y,
                                       int* status, void* stream) {
    if (n < 1 || n > MMF_NOALLOC_TRIDIAG_NMAX)
        return mmf_set_error(MMF_ERR_UNSUPPORTED,
                             "mmf_tridiag_eig_noalloc: n = " + std::to_string(n) + " outside 1.." +
                                 std::to_string(MMF_NOALLOC_TRIDIAG_NMAX) + " (fixed scratch size)");
    if (!d || !E || !Y || (n > 1 && !e)) return mmf_set_error(MMF_ERR_ARG, "d, e, E and Y are required");
    unsigned char* s = nullptr;
    int rc = scratch_for_current_device(&s);
    if (rc != MMF_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    MmfDesc* desc = (MmfDesc*)(s + NA_OFF_DESC);
    int* idx = (int*)(s + NA_OFF_INT);
    // the status word: the caller's, or one in the scratch array
    int* stw = status ? status : (int*)(s + NA_OFF_INT + sizeof(int));
    k_noalloc_setup<<<1, 32, 0, st>>>(desc, idx, stw, n);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess)
        return mmf_set_error(MMF_ERR_CUDA, std::string("mmf_tridiag_eig_noalloc set-up: ") + cudaGetErrorString(err));
    MmfLaunch L;
    L.desc = desc;
    L.idx = idx;
    L.count = 1;
    L.nmax = n;
    L.stream = st;
    err = mmf_launch_tridiag_eig(L, d, e, (double*)(s + NA_OFF_AUX), (double*)(s + NA_OFF_E2), E, Y,
                                 (double*)(s + NA_OFF_WORK), stw, 0, 3);
    if (err != cudaSuccess)
        return mmf_set_error(MMF_ERR_CUDA, std::string("mmf_tridiag_eig_noalloc: ") + cudaGetErrorString(err));
    return MMF_OK;
}
