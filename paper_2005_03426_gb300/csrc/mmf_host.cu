// mmf_host.cu -- host runtime behind the C ABI of include/mmf.h: contexts, system
// definitions, batch plans (device memory layout inside an HBM budget) and the launch
// sequence S1 assemble -> S2..S6 eigendecomposition -> S7 U(t, t0) -> S8 Pbar.
//
// Call sequence of the paper (Sec. 3.1-3.2, Fig. 2): define the system (levels, static part,
// modes and couplings), build the Floquet matrix, diagonalise, evaluate U / Pbar.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/mmf.h"
#include "mmf_internal.h"


static thread_local std::string g_last_error;
static thread_local int g_launches = 0;

static int fail(int code, const std::string& msg) {
    g_last_error = msg;
    return code;
}

// error reporting for the library's other host translation units
int mmf_set_error(int code, const std::string& msg) { return fail(code, msg); }

#define CU(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(MMF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// A tuning rule: for systems of one precision with n in [n_lo, n_hi] and half-bandwidth in
// [band_lo, band_hi], the solver choices (-1 = no preference: the context's thresholds decide).
struct TuneRule {
    int precision;
    int64_t n_lo, n_hi;
    int band_lo, band_hi;
    int jacobi, band, bt_tc;
};

struct mmf_ctx {
    int device = 0;
    std::vector<TuneRule> rules;     // first match wins
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t budget = 0, used = 0;
    int64_t jacobi_n[2] = {-1, -1};  // per precision; -1 = library default
    int64_t large_n = -1;            // whole-GPU reduction from this n on; -1 = when one CTA cannot
    int64_t refine_full_n = -1;      // mixed path: second refinement step in full from this n on
    int64_t gram_kernel = 0;         // mixed path: 0 = BF16 tensor cores (exact slicing), 1 = double-FP32
    int64_t bt_tc_n = -1;            // mixed path: back-transform on the tensor cores from this n on
    int64_t jacobi_sweeps = -1;      // Jacobi sweep cap; -1 = library default
    int64_t band_max = -1;           // largest half-bandwidth reduced by the bulge chase; -1 = default
    int64_t hetrd_tc = -1;           // mixed path: dense reduction's trailing update on the tensor cores
    cudaEvent_t order_ev = nullptr;  // orders the context stream against callers' streams (*_dev calls)
    std::recursive_mutex mu;
};

struct mmf_sys {
    mmf_ctx* ctx = nullptr;
    int D = 0;
    std::vector<double2> H0;
    std::vector<double> omega;
    std::vector<int> N;
    std::vector<std::vector<std::vector<double2>>> V;  // [mode][harmonic-1][D*D]
    mmf_batch* solo = nullptr;
    int state = 0;  // 0 defined, 1 built, 2 diagonalised
};

struct Pool {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = (off + 255) & ~(size_t)255;
        off = o + bytes;
        return o;
    }
};

struct mmf_batch {
    mmf_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;  // the context's stream, or a serving slot's stream
    int count = 0, precision = 0, nt = 0;
    std::vector<mmf_sys*> sys;
    std::vector<MmfDesc> desc;
    std::vector<int> all, small, large, medium, huge;  // large = medium + huge + the banded ones
    // banded systems reduced by the bulge chase, per window class (8, 16, 32, 64)
    std::vector<int> sbr[4];
    int nmax_sbr[4] = {0, 0, 0, 0};
    int* d_sbr[4] = {nullptr, nullptr, nullptr, nullptr};
    // band back-transform: per window class on the FP32 / FP64 units ([0..3]), on the tensor cores ([4])
    std::vector<int> sbt[5];
    int nmax_sbt[5] = {0, 0, 0, 0, 0};
    int* d_sbt[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    std::vector<int> rband, rfull;                     // mixed: hybrid / full second refinement step
    std::vector<int> btc, bts;                         // large: back-transform on tensor cores / SIMT
    std::vector<int> btc_n;                            // n of each system in btc
    int nmax_btc = 0, nmax_bts = 0;
    int *d_btc = nullptr, *d_bts = nullptr;
    void* d_btjobs = nullptr;                          // 4 x count Tf3Job
    int nmax_rband = 0, nmax_rfull = 0;
    int nmax_all = 0, nmax_small = 0, nmax_large = 0, Mmax = 1, Dmax = 1;
    int64_t n_oz = 0;      // BF16 elements of the Gram-product slices (mixed, tensor-core Gram)
    int gram_kernel = 0;   // copied from the context at creation
    int jacobi_sweeps = 40;  // copied from the context at creation
    int hetrd_tc = 1;        // copied from the context at creation
    int64_t n_pat = 0;
    int* d_pat = nullptr;  // mixed path: nonzero pattern of the coefficient rows
    int64_t n_coef = 0, n_mat = 0, n_vec = 0, n_sq = 0, n_pan = 0, n_t = 0, n_f = 0, n_u = 0,
            n_p = 0;
    // device
    unsigned char* base = nullptr;
    size_t bytes = 0;
    MmfDesc* d_desc = nullptr;
    int *d_all = nullptr, *d_small = nullptr, *d_large = nullptr, *d_medium = nullptr, *d_status = nullptr;
    int *d_rband = nullptr, *d_rfull = nullptr;
    int nmax_medium = 0;
    double2* d_coef = nullptr;
    void* d_H = nullptr;
    double2* d_Zf = nullptr;
    void* d_Zp = nullptr;
    double *d_E = nullptr, *d_d = nullptr, *d_e = nullptr, *d_e2 = nullptr, *d_aux = nullptr;
    void* d_tau = nullptr;
    double *d_Y = nullptr, *d_work = nullptr;
    void *d_Vp = nullptr, *d_Wp = nullptr;
    double* d_t = nullptr;
    double2 *d_F = nullptr, *d_U = nullptr;
    double* d_P = nullptr;
    double2 *d_R = nullptr, *d_S = nullptr, *d_HX = nullptr, *d_Eb = nullptr, *d_T = nullptr;
    float2* d_X1 = nullptr;
    float4* d_coefs = nullptr;  // coefficients split into FP32 pieces (mixed refinement)
    void* d_oz = nullptr;       // Gram-product slices (BF16)
    int* d_ozexp = nullptr;     // per-column scale exponents of the slices
    float2* d_Zs = nullptr;     // FP64 path: Z split into FP32 pieces for the time evolution
    double* d_E2 = nullptr;
    int* d_cid = nullptr;
    void* d_jobs = nullptr;
    // host staging (pinned)
    double2* h_coef = nullptr;
    double* h_t = nullptr;
    double t0 = 0.0;
    bool pinned = true;     // host staging buffers page-locked (false: pageable, for serving)
    bool times_set = false;
    int last_stage = 0;  // 1 assembled, 2 diagonalised, 3 outputs
    // per-stage CUDA-event timing (optional)
    int timing_runs = 0, runs_recorded = 0;
    std::vector<cudaEvent_t> ev;
    // CUDA graph of the whole run (optional)
    bool use_graph = false;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_launches = 0;
};

enum { ST_ASSEMBLE, ST_JACOBI, ST_HETRD, ST_TRIDIAG, ST_BACKTRANSFORM, ST_REFINE, ST_GRAM, ST_REFINE2,
       ST_OUTPUTS, ST_COUNT };

static void mark(mmf_batch* b, int stage) {
    if (b->timing_runs <= 0) return;
    int slot = b->runs_recorded % b->timing_runs;
    cudaEventRecord(b->ev[(size_t)slot * (ST_COUNT + 1) + stage], b->stream);
}

// ------------------------------------------------------------------ helpers
static int64_t round_up(int64_t v, int64_t m) { return (v + m - 1) / m * m; }

static int jacobi_default(int prec) { return prec == MMF_MIXED ? MMF_JACOBI_NMAX_F32 : MMF_JACOBI_NMAX_F64; }
static int jacobi_nmax(const mmf_ctx* c, int prec) {
    const int64_t v = c ? c->jacobi_n[prec == MMF_MIXED] : -1;
    // systems with n <= 4 always take the Jacobi kernel (the tridiagonal solver's FP32 work layout
    // assumes n >= 4)
    return v < 0 ? jacobi_default(prec) : (int)std::max<int64_t>(4, std::min<int64_t>(v, jacobi_default(prec)));
}

static int64_t bt_tc_n(const mmf_ctx* c) {
    return (c && c->bt_tc_n >= 0) ? c->bt_tc_n : (int64_t)MMF_BT_TC_NMIN;
}
static int64_t refine_full_n(const mmf_ctx* c) {
    return (c && c->refine_full_n >= 0) ? c->refine_full_n : (int64_t)MMF_REFINE_FULL2_N;
}

static int64_t sys_dim(const mmf_sys* s) {
    int64_t m = 1;
    for (int N : s->N) m *= (2 * N + 1);
    return (int64_t)s->D * m;
}

// Half-bandwidth of H_F (Eq. 6, Appendix A): the largest |row - col| of a nonzero entry.  H0
// contributes |i - i'|; harmonic h of mode l (present in H_F only if h <= 2 N_l) puts V^{l,h}
// at block offset h S_l, so its entry (i, i') lands at column - row = D h S_l + i' - i.
static int sys_band(const mmf_sys* s) {
    const int D = s->D;
    int64_t b = 0;
    for (int i = 0; i < D; ++i)
        for (int k = 0; k < D; ++k) {
            const double2 h = s->H0[(size_t)i * D + k];
            if (h.x != 0.0 || h.y != 0.0) b = std::max<int64_t>(b, std::abs(i - k));
        }
    int64_t S = 1;
    for (size_t l = 0; l < s->omega.size(); ++l) {
        for (size_t h = 0; h < s->V[l].size() && (int64_t)(h + 1) <= 2 * (int64_t)s->N[l]; ++h) {
            const auto& V = s->V[l][h];
            for (int i = 0; i < D; ++i)
                for (int k = 0; k < D; ++k) {
                    const double2 v = V[(size_t)i * D + k];
                    if (v.x != 0.0 || v.y != 0.0) b = std::max<int64_t>(b, (int64_t)D * (int64_t)(h + 1) * S + k - i);
                }
        }
        S *= 2 * (int64_t)s->N[l] + 1;
    }
    return (int)std::min<int64_t>(std::max<int64_t>(b, 1), INT32_MAX / 4);
}

// Spin couplings of Eq. 7 (host only).  S_z = diag(m), S_+ |m> = sqrt(S(S+1) - m(m+1)) |m+1>,
// S_x = (S_+ + S_-)/2, S_y = (S_+ - S_-)/(2i), in the basis m = S, S-1, ..., -S.
extern "C" int mmf_spin_components(int S2, const double* A, const double* phi, int is_static, double* V) {
    if (S2 < 1 || !A || !V || (!is_static && !phi)) return fail(MMF_ERR_ARG, "spin components: S2 >= 1, A, phi, V required");
    const int D = S2 + 1;
    const double S = 0.5 * S2;
    // factor of each Cartesian component: A_i (static) or (A_i / 2) e^{i phi_i} (drive)
    double cr[3], ci[3];
    for (int k = 0; k < 3; ++k) {
        if (is_static) {
            cr[k] = A[k];
            ci[k] = 0.0;
        } else {
            cr[k] = 0.5 * A[k] * std::cos(phi[k]);
            ci[k] = 0.5 * A[k] * std::sin(phi[k]);
        }
    }
    for (int e = 0; e < 2 * D * D; ++e) V[e] = 0.0;
    for (int r = 0; r < D; ++r) {
        const double m = S - r;  // row r holds <m|
        // S_z
        V[2 * (r * D + r)] += cr[2] * m;
        V[2 * (r * D + r) + 1] += ci[2] * m;
        // <m| S_+ |m-1> = sqrt(S(S+1) - (m-1) m): column r + 1 holds |m - 1>
        if (r + 1 < D) {
            const double s = std::sqrt(S * (S + 1.0) - (m - 1.0) * m);
            // <m|S_x|m-1> = s/2, <m|S_y|m-1> = s/(2i) = -i s/2 ; <m-1|S_x|m> = s/2, <m-1|S_y|m> = i s/2
            const double hx = 0.5 * s;
            // upper entry (r, r+1): cx * hx + cy * (-i hx)
            V[2 * (r * D + r + 1)] += cr[0] * hx + ci[1] * hx;
            V[2 * (r * D + r + 1) + 1] += ci[0] * hx - cr[1] * hx;
            // lower entry (r+1, r): cx * hx + cy * (i hx)
            V[2 * ((r + 1) * D + r)] += cr[0] * hx - ci[1] * hx;
            V[2 * ((r + 1) * D + r) + 1] += ci[0] * hx + cr[1] * hx;
        }
    }
    return MMF_OK;
}

extern "C" const char* mmf_strerror(int st) {
    switch (st) {
        case MMF_OK: return "ok";
        case MMF_ERR_ARG: return "invalid argument";
        case MMF_ERR_STATE: return "call out of order";
        case MMF_ERR_BUDGET: return "request exceeds the context's HBM budget";
        case MMF_ERR_CUDA: return "CUDA error";
        case MMF_ERR_UNSUPPORTED: return "unsupported size or option";
        case MMF_ERR_NOMEM: return "host allocation failed";
        case MMF_ST_NOCONV: return "iteration cap reached";
        case MMF_ST_NONFINITE: return "non-finite value";
        case MMF_ST_CLUSTER: return "cluster of close eigenvalues too large to separate";
        default: return "unknown status";
    }
}
extern "C" const char* mmf_last_error(void) { return g_last_error.c_str(); }
extern "C" int mmf_last_launch_count(void) { return g_launches; }

// ------------------------------------------------------------------ context
extern "C" int mmf_ctx_create(int device, size_t budget, void* stream, mmf_ctx** out) {
    if (!out) return fail(MMF_ERR_ARG, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    CU(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(MMF_ERR_ARG, "no such CUDA device");
    CU(cudaSetDevice(device));
    mmf_ctx* c = new (std::nothrow) mmf_ctx();
    if (!c) return fail(MMF_ERR_NOMEM, "context allocation");
    c->device = device;
    if (stream) {
        c->stream = (cudaStream_t)stream;
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(MMF_ERR_CUDA, cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    // keep freed batch memory in the stream-ordered pool of this process for reuse
    cudaMemPool_t pool;
    uint64_t pool_idle = 0;  // reserved by the pool but not in use: available to new batches
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        uint64_t reserved = 0, used = 0;
        if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
            pool_idle = reserved - used;
    }
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            if (c->own_stream) cudaStreamDestroy(c->stream);
            delete c;
            return fail(MMF_ERR_CUDA, cudaGetErrorString(e));
        }
        budget = (fr + (size_t)pool_idle) / 10 * 9;
    }
    c->budget = budget;
    *out = c;
    return MMF_OK;
}

extern "C" int mmf_ctx_destroy(mmf_ctx* c) {
    if (!c) return MMF_ERR_ARG;
    cudaSetDevice(c->device);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    if (c->order_ev) cudaEventDestroy(c->order_ev);
    delete c;
    return MMF_OK;
}
extern "C" size_t mmf_ctx_bytes_in_use(const mmf_ctx* c) { return c ? c->used : 0; }

extern "C" int mmf_ctx_set_option(mmf_ctx* c, int option, int64_t value) {
    if (!c) return fail(MMF_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    switch (option) {
        case MMF_OPT_JACOBI_N_FP64: c->jacobi_n[0] = value; return MMF_OK;
        case MMF_OPT_JACOBI_N_MIXED: c->jacobi_n[1] = value; return MMF_OK;
        case MMF_OPT_LARGE_N: c->large_n = value; return MMF_OK;
        case MMF_OPT_REFINE_FULL_N: c->refine_full_n = value; return MMF_OK;
        case MMF_OPT_BT_TC_N: c->bt_tc_n = value; return MMF_OK;
        case MMF_OPT_JACOBI_SWEEPS: c->jacobi_sweeps = value; return MMF_OK;
        case MMF_OPT_BAND_MAX: c->band_max = value; return MMF_OK;
        case MMF_OPT_HETRD_TC: c->hetrd_tc = value; return MMF_OK;
        case MMF_OPT_GRAM_KERNEL:
            if (value > 1) return fail(MMF_ERR_ARG, "MMF_OPT_GRAM_KERNEL: 0 (tensor cores) or 1 (double-FP32)");
            c->gram_kernel = value < 0 ? 0 : value;
            return MMF_OK;
        default: return fail(MMF_ERR_ARG, "unknown option");
    }
}
extern "C" size_t mmf_ctx_budget(const mmf_ctx* c) { return c ? c->budget : 0; }

extern "C" int mmf_ctx_add_rule(mmf_ctx* c, int precision, int64_t n_lo, int64_t n_hi, int band_lo, int band_hi,
                                int jacobi, int band, int bt_tc) {
    if (!c) return fail(MMF_ERR_ARG, "ctx is NULL");
    if (precision != MMF_FP64 && precision != MMF_MIXED) return fail(MMF_ERR_ARG, "bad precision");
    if (n_lo > n_hi || band_lo > band_hi) return fail(MMF_ERR_ARG, "empty rule range");
    if (jacobi < -1 || jacobi > 1 || band < -1 || band > 1 || bt_tc < -1 || bt_tc > 1)
        return fail(MMF_ERR_ARG, "rule choices are -1, 0 or 1");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    c->rules.push_back({precision, n_lo, n_hi, band_lo, band_hi, jacobi, band, bt_tc});
    return MMF_OK;
}

extern "C" int mmf_ctx_clear_rules(mmf_ctx* c) {
    if (!c) return fail(MMF_ERR_ARG, "ctx is NULL");
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    c->rules.clear();
    return MMF_OK;
}

extern "C" int mmf_ctx_load_tuning(mmf_ctx* c, const char* path) {
    if (!c || !path) return fail(MMF_ERR_ARG, "ctx and path required");
    FILE* f = std::fopen(path, "r");
    if (!f) return fail(MMF_ERR_ARG, std::string("cannot open tuning table ") + path);
    char line[512];
    int ln = 0, added = 0;
    std::vector<TuneRule> rules;
    while (std::fgets(line, sizeof(line), f)) {
        ++ln;
        char* p = line;
        while (*p == ' ' || *p == '\t') ++p;
        if (*p == '#' || *p == '\n' || *p == '\0') continue;
        char prec[16];
        long long nlo, nhi;
        int blo, bhi, jac, bnd, btc;
        if (std::sscanf(p, "%15s %lld %lld %d %d %d %d %d", prec, &nlo, &nhi, &blo, &bhi, &jac, &bnd, &btc) != 8) {
            std::fclose(f);
            return fail(MMF_ERR_ARG, std::string(path) + ":" + std::to_string(ln) + ": expected 8 fields");
        }
        const std::string ps(prec);
        if (ps != "fp64" && ps != "mixed") {
            std::fclose(f);
            return fail(MMF_ERR_ARG, std::string(path) + ":" + std::to_string(ln) + ": precision fp64 or mixed");
        }
        if (nlo > nhi || blo > bhi || jac < -1 || jac > 1 || bnd < -1 || bnd > 1 || btc < -1 || btc > 1) {
            std::fclose(f);
            return fail(MMF_ERR_ARG, std::string(path) + ":" + std::to_string(ln) + ": bad range or choice");
        }
        rules.push_back({ps == "fp64" ? MMF_FP64 : MMF_MIXED, (int64_t)nlo, (int64_t)nhi, blo, bhi, jac, bnd, btc});
        ++added;
    }
    std::fclose(f);
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    c->rules.insert(c->rules.end(), rules.begin(), rules.end());
    return added;
}

// ------------------------------------------------------------------ systems
extern "C" int mmf_sys_create(mmf_ctx* ctx, int D, const double* H0, mmf_sys** out) {
    if (!out) return fail(MMF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || D < 1 || !H0) return fail(MMF_ERR_ARG, "ctx, D >= 1 and H0 required");
    double mx = 0.0;
    for (int i = 0; i < 2 * D * D; ++i) {
        if (!std::isfinite(H0[i])) return fail(MMF_ST_NONFINITE, "H0 not finite");
        mx = std::max(mx, std::fabs(H0[i]));
    }
    for (int i = 0; i < D; ++i)
        for (int j = 0; j < D; ++j) {
            double ar = H0[2 * (i * D + j)], ai = H0[2 * (i * D + j) + 1];
            double br = H0[2 * (j * D + i)], bi = H0[2 * (j * D + i) + 1];
            if (std::fabs(ar - br) > 1e-12 * mx || std::fabs(ai + bi) > 1e-12 * mx)
                return fail(MMF_ERR_ARG, "H0 is not Hermitian");
        }
    mmf_sys* s = new (std::nothrow) mmf_sys();
    if (!s) return fail(MMF_ERR_NOMEM, "system allocation");
    s->ctx = ctx;
    s->D = D;
    s->H0.resize((size_t)D * D);
    for (int e = 0; e < D * D; ++e) s->H0[e] = make_double2(H0[2 * e], H0[2 * e + 1]);
    *out = s;
    return MMF_OK;
}

extern "C" int mmf_add_mode(mmf_sys* s, double omega, int N, int* mode_id) {
    if (!s) return fail(MMF_ERR_ARG, "sys is NULL");
    if (!(omega > 0.0) || !std::isfinite(omega)) return fail(MMF_ERR_ARG, "omega must be > 0");
    if (N < 0) return fail(MMF_ERR_ARG, "N must be >= 0");
    if ((int)s->omega.size() >= MMF_MAX_MODES) return fail(MMF_ERR_UNSUPPORTED, "at most 4 modes");
    s->omega.push_back(omega);
    s->N.push_back(N);
    s->V.emplace_back();
    if (mode_id) *mode_id = (int)s->omega.size() - 1;
    s->state = 0;
    return MMF_OK;
}

extern "C" int mmf_add_coupling(mmf_sys* s, int mode_id, int harmonic, const double* V) {
    if (!s || !V) return fail(MMF_ERR_ARG, "sys and V required");
    if (mode_id < 0 || mode_id >= (int)s->omega.size()) return fail(MMF_ERR_ARG, "bad mode id");
    if (harmonic < 1) return fail(MMF_ERR_ARG, "harmonic must be >= 1");
    auto& hv = s->V[mode_id];
    if (harmonic > (int)hv.size() + 1) return fail(MMF_ERR_ARG, "harmonics must be added in order");
    std::vector<double2> m((size_t)s->D * s->D);
    for (int e = 0; e < s->D * s->D; ++e) {
        if (!std::isfinite(V[2 * e]) || !std::isfinite(V[2 * e + 1]))
            return fail(MMF_ST_NONFINITE, "V not finite");
        m[e] = make_double2(V[2 * e], V[2 * e + 1]);
    }
    if (harmonic == (int)hv.size() + 1) hv.push_back(m);
    else hv[harmonic - 1] = m;
    s->state = 0;
    return MMF_OK;
}

extern "C" int mmf_batch_destroy(mmf_batch* b);

extern "C" int mmf_sys_destroy(mmf_sys* s) {
    if (!s) return MMF_ERR_ARG;
    if (s->solo) mmf_batch_destroy(s->solo);
    delete s;
    return MMF_OK;
}

extern "C" int64_t mmf_dim(const mmf_sys* s) { return s ? sys_dim(s) : -1; }
extern "C" int mmf_sys_bandwidth(const mmf_sys* s) { return s ? sys_band(s) : -1; }

// ------------------------------------------------------------------ batch plan
static void fill_coef(const mmf_batch* b, double2* dst) {
    for (int i = 0; i < b->count; ++i) {
        const mmf_sys* s = b->sys[i];
        double2* p = dst + b->desc[i].coef_off;
        std::memcpy(p, s->H0.data(), sizeof(double2) * s->H0.size());
        p += s->H0.size();
        for (size_t l = 0; l < s->V.size(); ++l)
            for (const auto& m : s->V[l]) {
                std::memcpy(p, m.data(), sizeof(double2) * m.size());
                p += m.size();
            }
    }
}

static void free_batch_memory(mmf_batch* b) {
    if (b->base) {
        cudaFreeAsync(b->base, b->stream);
        b->ctx->used -= b->bytes;
        b->base = nullptr;
    }
    if (b->pinned) {
        if (b->h_coef) cudaFreeHost(b->h_coef);
        if (b->h_t) cudaFreeHost(b->h_t);
    } else {
        free(b->h_coef);
        free(b->h_t);
    }
    b->h_coef = nullptr;
    b->h_t = nullptr;
}

static int batch_create(mmf_ctx* ctx, int count, mmf_sys* const* systems, int precision, int nt,
                        cudaStream_t stream, bool pinned_staging, mmf_batch** out);

extern "C" int mmf_batch_create(mmf_ctx* ctx, int count, mmf_sys* const* systems, int precision,
                                int nt, mmf_batch** out) {
    return batch_create(ctx, count, systems, precision, nt, ctx ? ctx->stream : nullptr, true, out);
}

static int batch_create(mmf_ctx* ctx, int count, mmf_sys* const* systems, int precision, int nt,
                        cudaStream_t stream, bool pinned_staging, mmf_batch** out) {
    if (!out) return fail(MMF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || count < 1 || !systems || nt < 0) return fail(MMF_ERR_ARG, "bad batch arguments");
    if (precision != MMF_FP64 && precision != MMF_MIXED) return fail(MMF_ERR_ARG, "bad precision");
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    CU(cudaSetDevice(ctx->device));
    mmf_batch* b = new (std::nothrow) mmf_batch();
    if (!b) return fail(MMF_ERR_NOMEM, "batch allocation");
    b->ctx = ctx;
    b->stream = stream;
    b->pinned = pinned_staging;
    b->count = count;
    b->precision = precision;
    b->nt = nt;
    b->gram_kernel = (int)ctx->gram_kernel;
    b->jacobi_sweeps = ctx->jacobi_sweeps < 0 ? 40 : (int)std::max<int64_t>(1, std::min<int64_t>(ctx->jacobi_sweeps, 1000));
    b->hetrd_tc = ctx->hetrd_tc != 0;
    b->sys.assign(systems, systems + count);
    b->desc.resize(count);
    const int fp32 = precision == MMF_MIXED;
    const int hmax = mmf_hetrd_max_n(fp32);
    const int jmax = jacobi_nmax(ctx, precision);
    const int64_t lmin = ctx->large_n < 0 ? (int64_t)hmax + 1 : ctx->large_n;
    for (int i = 0; i < count; ++i) {
        const mmf_sys* s = systems[i];
        if (!s || s->ctx != ctx) { delete b; return fail(MMF_ERR_ARG, "system NULL or from another context"); }
        if (s->omega.empty()) { delete b; return fail(MMF_ERR_ARG, "system has no drive mode"); }
        MmfDesc& d = b->desc[i];
        std::memset(&d, 0, sizeof(d));
        d.D = s->D;
        d.K = (int)s->omega.size();
        int64_t M = 1, b0 = 0;
        for (int k = 0; k < d.K; ++k) {
            d.N[k] = s->N[k];
            d.S[k] = (int)M;
            b0 += (int64_t)s->N[k] * M;
            M *= (2 * s->N[k] + 1);
            d.omega[k] = s->omega[k];
            d.nharm[k] = (int)s->V[k].size();
        }
        int64_t n = M * s->D;
        if (n > (int64_t)INT32_MAX / 4) {
            delete b;
            return fail(MMF_ERR_UNSUPPORTED, "Floquet dimension " + std::to_string(n) + " too large");
        }
        d.M = (int)M;
        d.n = (int)n;
        d.b0 = (int)b0;
        d.ld = (int)round_up(std::max<int64_t>(n, MMF_MIN_LD), 4);
        // solver choices: a matching tuning rule, else the size thresholds
        const int band_raw = sys_band(s);
        const TuneRule* rule = nullptr;
        for (const TuneRule& ru : ctx->rules)
            if (ru.precision == precision && n >= ru.n_lo && n <= ru.n_hi && band_raw >= ru.band_lo &&
                band_raw <= ru.band_hi) {
                rule = &ru;
                break;
            }
        d.small = n <= jmax;
        if (rule && rule->jacobi >= 0) d.small = n <= 4 || (rule->jacobi && n <= jacobi_default(precision));
        int64_t nc = (int64_t)s->D * s->D;
        for (int k = 0; k < d.K; ++k) nc += (int64_t)d.nharm[k] * s->D * s->D;
        d.coef_off = b->n_coef;
        b->n_coef += nc;
        // sparse coefficient rows pay off in the refinement's H_F products from a few dozen levels
        d.pat_cap = (precision == MMF_MIXED && s->D >= 32) ? 16 : 0;
        d.pat_off = b->n_pat;
        b->n_pat += d.pat_cap ? 1 + (int64_t)coef_matrices(d) * s->D * (1 + d.pat_cap) : 1;
        d.mat_off = b->n_mat;
        b->n_mat += n * d.ld;
        d.vec_off = b->n_vec;
        b->n_vec += n;
        d.sq_off = b->n_sq;
        d.oz_off = b->n_oz;
        // banded systems: bulge chase instead of the dense reduction and its back-transform
        int64_t bmax_opt = ctx->band_max < 0 ? (precision == MMF_FP64 ? 64 : 0) : std::min<int64_t>(ctx->band_max, 64);
        if (rule && rule->band >= 0) bmax_opt = rule->band ? 64 : 0;
        int cls = 0;
        if (!d.small && bmax_opt > 0) {
            const int band = band_raw;
            if (band <= bmax_opt && n >= 2 * (int64_t)band + 2 && n * (int64_t)d.ld < INT32_MAX &&
                mmf_sbr_store_elems((int)n, band) <= n * (int64_t)d.ld) {
                d.band = band;
                cls = mmf_sbr_class(band);
            }
        }
        // mixed: back-transform on the tensor cores for large enough systems (SIMT otherwise); on
        // the band path for the widest window class when the blocks' T factors fit the work slot
        bool tc = precision == MMF_MIXED && !d.small && !cls && n >= std::max<int64_t>(bt_tc_n(ctx), 3);
        if (rule && rule->bt_tc >= 0) tc = precision == MMF_MIXED && !d.small && !cls && n >= 3 && rule->bt_tc;
        const bool band_tc_ok = precision == MMF_MIXED && cls == 64;
        bool band_tc = band_tc_ok && n >= bt_tc_n(ctx);
        if (rule && rule->bt_tc >= 0) band_tc = band_tc_ok && rule->bt_tc;
        if (precision == MMF_MIXED) {
            // one area per system, used in turn by the back-transform's operands, the Gram slices
            // (BF16) and split-TF32 operands of the refinement, and the time evolution's slices and Phi
            const int64_t oz = ctx->gram_kernel == 0 ? (int64_t)mmf_ozaki_slice_elems((int)n) : 0;
            const int64_t ph = (nt > 0 && s->D <= mmf_phi_max_levels() && M <= mmf_ozaki_max_n())
                                   ? mmf_phi_elems((int)n, s->D, (int)M, nt)
                                   : 0;
            const int64_t bt = tc ? 2 * mmf_bt_floats((int)n) : band_tc ? mmf_sbt_ops_elems((int)n, d.band) : 0;
            b->n_oz += std::max<int64_t>(std::max<int64_t>(oz, 2 * mmf_tf3_floats((int)n)), std::max<int64_t>(bt, ph));
        }
        if (cls) {
            const int ci = cls == 8 ? 0 : cls == 16 ? 1 : cls == 32 ? 2 : 3;
            b->sbr[ci].push_back(i);
            b->nmax_sbr[ci] = std::max(b->nmax_sbr[ci], (int)n);
            const int bi = band_tc ? 4 : ci;
            b->sbt[bi].push_back(i);
            b->nmax_sbt[bi] = std::max(b->nmax_sbt[bi], (int)n);
        } else if (!d.small) {
            (tc ? b->btc : b->bts).push_back(i);
            if (tc) {
                b->btc_n.push_back((int)n);
                b->nmax_btc = std::max(b->nmax_btc, (int)n);
            } else {
                b->nmax_bts = std::max(b->nmax_bts, (int)n);
            }
        }
        d.pan_off = b->n_pan;
        if (!d.small) {
            b->n_sq += n * n;
            b->n_pan += (int64_t)(d.ld + MMF_NB) * MMF_NB;
        }
        d.t_off = b->n_t;
        b->n_t += nt;
        d.f_off = b->n_f;
        b->n_f += (int64_t)nt * M;
        d.u_off = b->n_u;
        b->n_u += (int64_t)nt * s->D * s->D;
        d.p_off = b->n_p;
        b->n_p += (int64_t)s->D * s->D;
        b->all.push_back(i);
        (d.small ? b->small : b->large).push_back(i);
        if (!d.small && !cls) (n >= lmin ? b->huge : b->medium).push_back(i);
        b->nmax_all = std::max(b->nmax_all, (int)n);
        if (d.small) b->nmax_small = std::max(b->nmax_small, (int)n);
        else b->nmax_large = std::max(b->nmax_large, (int)n);
        if (!d.small && !cls && n < lmin) b->nmax_medium = std::max(b->nmax_medium, (int)n);
        b->Mmax = std::max(b->Mmax, (int)M);
        b->Dmax = std::max(b->Dmax, s->D);
        if (n >= refine_full_n(ctx)) {
            b->rfull.push_back(i);
            b->nmax_rfull = std::max(b->nmax_rfull, (int)n);
        } else {
            b->rband.push_back(i);
            b->nmax_rband = std::max(b->nmax_rband, (int)n);
        }
    }
    // device layout
    const size_t cs = fp32 ? sizeof(float2) : sizeof(double2);
    Pool p;
    size_t o_desc = p.take(sizeof(MmfDesc) * count);
    size_t o_all = p.take(sizeof(int) * count), o_small = p.take(sizeof(int) * count),
           o_large = p.take(sizeof(int) * count), o_medium = p.take(sizeof(int) * count),
           o_status = p.take(sizeof(int) * count), o_rband = p.take(sizeof(int) * count),
           o_rfull = p.take(sizeof(int) * count), o_sbr = p.take(sizeof(int) * count), o_sbt = p.take(sizeof(int) * count),
           o_btc = p.take(sizeof(int) * count),
           o_bts = p.take(sizeof(int) * count);
    size_t o_coef = p.take(sizeof(double2) * b->n_coef);
    size_t o_H = p.take(cs * b->n_mat);
    size_t o_Zf = p.take(sizeof(double2) * b->n_mat);
    size_t o_E = p.take(sizeof(double) * b->n_vec), o_d = p.take(sizeof(double) * b->n_vec),
           o_e = p.take(sizeof(double) * b->n_vec), o_e2 = p.take(sizeof(double) * b->n_vec),
           o_aux = p.take(sizeof(double) * 8 * count);
    size_t o_tau = p.take(cs * b->n_vec);
    size_t o_Y = p.take(sizeof(double) * b->n_sq), o_work = p.take(sizeof(double) * 3 * b->n_sq);
    size_t o_Vp = p.take(cs * b->n_pan), o_Wp = p.take(cs * b->n_pan);
    size_t o_t = p.take(sizeof(double) * std::max<int64_t>(b->n_t, 1));
    size_t o_F = p.take(sizeof(double2) * std::max<int64_t>(b->n_f, 1));
    size_t o_U = p.take(sizeof(double2) * std::max<int64_t>(b->n_u, 1));
    size_t o_P = p.take(sizeof(double) * b->n_p);
    size_t o_pat = 0;
    size_t o_R = 0, o_S = 0, o_HX = 0, o_E2 = 0, o_cid = 0, o_jobs = 0, o_Eb = 0, o_T = 0, o_X1 = 0, o_coefs = 0, o_oz = 0,
           o_ozexp = 0;
    const size_t o_Zs = (!fp32 && nt > 0) ? p.take(sizeof(float2) * 2 * b->n_mat) : 0;
    if (fp32) {
        o_Eb = p.take(sizeof(double2) * b->n_vec * MMF_REFINE_BW);
        o_T = p.take(sizeof(double2) * b->n_mat);
        o_X1 = p.take(sizeof(float2) * b->n_mat);
        o_coefs = p.take(sizeof(float4) * std::max<int64_t>(b->n_coef, 1));
        o_oz = p.take(sizeof(uint16_t) * std::max<int64_t>(b->n_oz, 1));
        o_ozexp = p.take(sizeof(int) * b->n_vec);
        o_R = p.take(sizeof(double2) * b->n_mat);
        o_S = p.take(sizeof(double2) * b->n_mat);
        o_HX = p.take(sizeof(double2) * b->n_mat);
        o_E2 = p.take(sizeof(double) * b->n_vec);
        o_cid = p.take(sizeof(int) * b->n_vec);
        o_jobs = p.take(std::max(sizeof(UmmaJob), sizeof(Tf3Job)) * count);
        o_pat = p.take(sizeof(int) * std::max<int64_t>(b->n_pat, 1));
    }
    const size_t o_btjobs = b->btc.empty() ? 0 : p.take(sizeof(Tf3Job) * 4 * b->btc.size());
    b->bytes = p.off;
    if (ctx->used + b->bytes > ctx->budget) {
        size_t need = b->bytes;
        const int64_t b_nmat = b->n_mat, b_noz = b->n_oz, b_nmax = b->nmax_all;
        delete b;
        return fail(MMF_ERR_BUDGET, "batch needs " + std::to_string(need) + " bytes, budget has " +
                                        std::to_string(ctx->budget - ctx->used) + " (elements: matrices " +
                                        std::to_string(b_nmat) + ", operand area " + std::to_string(b_noz) +
                                        ", largest n " + std::to_string(b_nmax) + ")");
    }
    cudaError_t e = cudaMallocAsync((void**)&b->base, b->bytes, b->stream);
    if (e == cudaErrorMemoryAllocation) {
        // memory other contexts of this process freed may sit idle in the pool: release it, retry
        cudaGetLastError();
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
            cudaStreamSynchronize(b->stream);
            cudaMemPoolTrimTo(pool, 0);
        }
        e = cudaMallocAsync((void**)&b->base, b->bytes, b->stream);
    }
    if (e != cudaSuccess) {
        delete b;
        return fail(MMF_ERR_CUDA, std::string("cudaMallocAsync: ") + cudaGetErrorString(e));
    }
    ctx->used += b->bytes;
    unsigned char* B = b->base;
    b->d_desc = (MmfDesc*)(B + o_desc);
    b->d_all = (int*)(B + o_all);
    b->d_small = (int*)(B + o_small);
    b->d_large = (int*)(B + o_large);
    b->d_medium = (int*)(B + o_medium);
    b->d_status = (int*)(B + o_status);
    b->d_rband = (int*)(B + o_rband);
    b->d_rfull = (int*)(B + o_rfull);
    b->d_btc = (int*)(B + o_btc);
    b->d_bts = (int*)(B + o_bts);
    {  // the four window classes share one index array, one after another
        int* q = (int*)(B + o_sbr);
        for (int ci = 0; ci < 4; ++ci) {
            b->d_sbr[ci] = q;
            q += b->sbr[ci].size();
        }
        int* qt = (int*)(B + o_sbt);
        for (int ci = 0; ci < 5; ++ci) {
            b->d_sbt[ci] = qt;
            qt += b->sbt[ci].size();
        }
    }
    if (!b->btc.empty()) b->d_btjobs = B + o_btjobs;
    b->d_coef = (double2*)(B + o_coef);
    b->d_H = B + o_H;
    b->d_Zf = (double2*)(B + o_Zf);
    // the FP32 back-transform output lives in HX, which the refinement only uses after widening
    b->d_Zp = fp32 ? (void*)(B + o_HX) : (void*)b->d_Zf;
    b->d_E = (double*)(B + o_E);
    b->d_d = (double*)(B + o_d);
    b->d_e = (double*)(B + o_e);
    b->d_e2 = (double*)(B + o_e2);
    b->d_aux = (double*)(B + o_aux);
    b->d_tau = B + o_tau;
    b->d_Y = (double*)(B + o_Y);
    b->d_work = (double*)(B + o_work);
    b->d_Vp = B + o_Vp;
    b->d_Wp = B + o_Wp;
    b->d_t = (double*)(B + o_t);
    b->d_F = (double2*)(B + o_F);
    b->d_U = (double2*)(B + o_U);
    b->d_P = (double*)(B + o_P);
    if (!fp32 && nt > 0) b->d_Zs = (float2*)(B + o_Zs);
    if (fp32) {
        b->d_R = (double2*)(B + o_R);
        b->d_S = (double2*)(B + o_S);
        b->d_HX = (double2*)(B + o_HX);
        b->d_E2 = (double*)(B + o_E2);
        b->d_cid = (int*)(B + o_cid);
        b->d_jobs = B + o_jobs;
        b->d_Eb = (double2*)(B + o_Eb);
        b->d_T = (double2*)(B + o_T);
        b->d_X1 = (float2*)(B + o_X1);
        b->d_coefs = (float4*)(B + o_coefs);
        b->d_oz = B + o_oz;
        b->d_ozexp = (int*)(B + o_ozexp);
        b->d_pat = (int*)(B + o_pat);
    }
    if (b->pinned) {
        e = cudaMallocHost((void**)&b->h_coef, sizeof(double2) * std::max<int64_t>(b->n_coef, 1));
        if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_t, sizeof(double) * std::max<int64_t>(b->n_t, 1));
    } else {
        b->h_coef = (double2*)malloc(sizeof(double2) * std::max<int64_t>(b->n_coef, 1));
        b->h_t = (double*)malloc(sizeof(double) * std::max<int64_t>(b->n_t, 1));
        e = (b->h_coef && b->h_t) ? cudaSuccess : cudaErrorMemoryAllocation;
    }
    if (e != cudaSuccess) {
        free_batch_memory(b);
        delete b;
        return fail(MMF_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    }
    fill_coef(b, b->h_coef);
    std::memset(b->h_t, 0, sizeof(double) * std::max<int64_t>(b->n_t, 1));
    cudaStream_t st = b->stream;
    e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(MmfDesc) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_all, b->all.data(), sizeof(int) * b->all.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->small.empty())
        e = cudaMemcpyAsync(b->d_small, b->small.data(), sizeof(int) * b->small.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->large.empty())
        e = cudaMemcpyAsync(b->d_large, b->large.data(), sizeof(int) * b->large.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->medium.empty())
        e = cudaMemcpyAsync(b->d_medium, b->medium.data(), sizeof(int) * b->medium.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->rband.empty())
        e = cudaMemcpyAsync(b->d_rband, b->rband.data(), sizeof(int) * b->rband.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->rfull.empty())
        e = cudaMemcpyAsync(b->d_rfull, b->rfull.data(), sizeof(int) * b->rfull.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->btc.empty())
        e = cudaMemcpyAsync(b->d_btc, b->btc.data(), sizeof(int) * b->btc.size(), cudaMemcpyHostToDevice, st);
    for (int ci = 0; ci < 4; ++ci)
        if (e == cudaSuccess && !b->sbr[ci].empty())
            e = cudaMemcpyAsync(b->d_sbr[ci], b->sbr[ci].data(), sizeof(int) * b->sbr[ci].size(),
                                cudaMemcpyHostToDevice, st);
    for (int ci = 0; ci < 5; ++ci)
        if (e == cudaSuccess && !b->sbt[ci].empty())
            e = cudaMemcpyAsync(b->d_sbt[ci], b->sbt[ci].data(), sizeof(int) * b->sbt[ci].size(),
                                cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !b->bts.empty())
        e = cudaMemcpyAsync(b->d_bts, b->bts.data(), sizeof(int) * b->bts.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_coef, b->h_coef, sizeof(double2) * b->n_coef, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        free_batch_memory(b);
        delete b;
        return fail(MMF_ERR_CUDA, std::string("upload: ") + cudaGetErrorString(e));
    }
    *out = b;
    return MMF_OK;
}

static void drop_events(mmf_batch* b) {
    for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
    b->ev.clear();
    b->timing_runs = 0;
    b->runs_recorded = 0;
}

extern "C" int mmf_batch_timing(mmf_batch* b, int max_runs) {
    if (!b || max_runs < 0 || max_runs > 4096) return fail(MMF_ERR_ARG, "bad batch or max_runs");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    CU(cudaStreamSynchronize(b->stream));
    drop_events(b);
    if (b->graph_exec) {  // the graph holds the old events
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    b->ev.resize((size_t)max_runs * (ST_COUNT + 1));
    for (auto& e : b->ev) CU(cudaEventCreate(&e));
    b->timing_runs = max_runs;
    return MMF_OK;
}

extern "C" int mmf_batch_stage_ms(mmf_batch* b, double* ms, int* runs) {
    if (!b || !ms) return fail(MMF_ERR_ARG, "batch and ms required");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    CU(cudaStreamSynchronize(b->stream));
    for (int s = 0; s < ST_COUNT; ++s) ms[s] = 0.0;
    int nr = std::min(b->runs_recorded, b->timing_runs);
    for (int r = 0; r < nr; ++r)
        for (int s = 0; s < ST_COUNT; ++s) {
            float f = 0.f;
            CU(cudaEventElapsedTime(&f, b->ev[(size_t)r * (ST_COUNT + 1) + s],
                                    b->ev[(size_t)r * (ST_COUNT + 1) + s + 1]));
            ms[s] += f;
        }
    if (runs) *runs = nr;
    b->runs_recorded = 0;
    return MMF_OK;
}

extern "C" int mmf_batch_destroy(mmf_batch* b) {
    if (!b) return MMF_ERR_ARG;
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    cudaSetDevice(b->ctx->device);
    cudaStreamSynchronize(b->stream);
    if (b->graph_exec) cudaGraphExecDestroy(b->graph_exec);
    drop_events(b);
    free_batch_memory(b);
    delete b;
    return MMF_OK;
}

extern "C" size_t mmf_batch_bytes(const mmf_batch* b) { return b ? b->bytes : 0; }

extern "C" int mmf_batch_set_times(mmf_batch* b, double t0, const double* t) {
    if (!b || (b->nt > 0 && !t)) return fail(MMF_ERR_ARG, "batch and times required");
    for (int64_t i = 0; i < b->n_t; ++i)
        if (!std::isfinite(t[i])) return fail(MMF_ST_NONFINITE, "time not finite");
    if (!std::isfinite(t0)) return fail(MMF_ST_NONFINITE, "t0 not finite");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaStreamSynchronize(b->stream));  // staging buffer may be in flight
    if (b->n_t > 0) std::memcpy(b->h_t, t, sizeof(double) * b->n_t);
    if (t0 != b->t0 && b->graph_exec) {  // t0 is a kernel argument baked into the graph
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    b->t0 = t0;
    b->times_set = true;
    if (b->n_t > 0)
        CU(cudaMemcpyAsync(b->d_t, b->h_t, sizeof(double) * b->n_t, cudaMemcpyHostToDevice, b->stream));
    return MMF_OK;
}

extern "C" int mmf_batch_upload(mmf_batch* b) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    cudaStream_t st = b->stream;
    CU(cudaMemcpyAsync(b->d_coef, b->h_coef, sizeof(double2) * b->n_coef, cudaMemcpyHostToDevice, st));
    if (b->n_t > 0)
        CU(cudaMemcpyAsync(b->d_t, b->h_t, sizeof(double) * b->n_t, cudaMemcpyHostToDevice, st));
    return MMF_OK;
}

static MmfLaunch launch_of(const mmf_batch* b, const std::vector<int>& list, const int* dlist, int nmax) {
    MmfLaunch L;
    L.desc = b->d_desc;
    L.idx = dlist;
    L.count = (int)list.size();
    L.nmax = nmax;
    L.stream = b->stream;
    return L;
}

#define LAUNCH(call, nk)                                                                  \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(MMF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        g_launches += (nk);                                                               \
    } while (0)

static int stage_assemble(mmf_batch* b) {
    const int fp32 = b->precision == MMF_MIXED;
    cudaStream_t st = b->stream;
    mark(b, ST_ASSEMBLE);
    CU(cudaMemsetAsync(b->d_status, 0, sizeof(int) * b->count, st));
    MmfLaunch La = launch_of(b, b->all, b->d_all, b->nmax_all);
    LAUNCH(mmf_launch_assemble(La, b->d_coef, b->d_H, fp32), 1);
    b->last_stage = 1;
    return MMF_OK;
}

// G = X1^H X1 (+ C' + C'^H in a second full step): BF16 tensor cores with exact slicing, or
// double-FP32 on the FP32 pipes
static cudaError_t refine_gram(mmf_batch* b, const MmfLaunch& L, int second) {
    if (b->gram_kernel == 0 && L.nmax <= mmf_ozaki_max_n()) {
        cudaError_t e = mmf_launch_ozaki_gram(L, b->d_X1, b->d_oz, b->d_ozexp, b->d_R, b->d_status);
        if (e != cudaSuccess || !second) return e;
        return mmf_launch_refine_gram_fix(L, b->d_R, b->d_T);
    }
    return mmf_launch_refine_gram(L, b->d_X1, b->d_R, b->d_T, second);
}

static int stage_eig(mmf_batch* b) {
    const int fp32 = b->precision == MMF_MIXED;
    mark(b, ST_JACOBI);
    if (!b->small.empty()) {
        MmfLaunch Ls = launch_of(b, b->small, b->d_small, b->nmax_small);
        LAUNCH(mmf_launch_jacobi(Ls, b->d_H, nullptr, b->d_E, b->d_Zf, b->d_status, fp32, b->jacobi_sweeps), 1);
    }
    if (!b->large.empty()) {
        MmfLaunch Ll = launch_of(b, b->large, b->d_large, b->nmax_large);
        mark(b, ST_HETRD);
        if (!b->medium.empty()) {
            MmfLaunch Lm = launch_of(b, b->medium, b->d_medium, b->nmax_medium);
            LAUNCH(mmf_launch_hetrd(Lm, b->d_H, b->d_Vp, b->d_Wp, b->d_d, b->d_e, b->d_tau, fp32, b->hetrd_tc,
                                    b->d_status),
                   1);
        }
        for (int ci = 0; ci < 4; ++ci) {  // banded systems: bulge chase
            if (b->sbr[ci].empty()) continue;
            MmfLaunch Lb = launch_of(b, b->sbr[ci], b->d_sbr[ci], b->nmax_sbr[ci]);
            LAUNCH(mmf_launch_sbr_chase(Lb, 8 << ci, b->d_H, b->d_Zf, b->d_d, b->d_e, b->d_status, fp32), 1);
        }
        for (int i : b->huge) {  // one system at a time over the whole GPU
            const MmfDesc& d = b->desc[i];
            void* work = (void*)(b->d_Y + d.sq_off);
            void* sc = (void*)(b->d_aux + 8 * i);
            LAUNCH(mmf_launch_hetrd_large(d, b->d_H, b->d_Vp, b->d_Wp, b->d_d, b->d_e, b->d_tau, work, sc, fp32,
                                          b->stream),
                   6 * d.n + (d.n + MMF_NB - 1) / MMF_NB);
        }
        mark(b, ST_TRIDIAG);
        LAUNCH(mmf_launch_tridiag_eig(Ll, b->d_d, b->d_e, b->d_aux, b->d_e2, b->d_E, b->d_Y, b->d_work,
                                      b->d_status, fp32, 3), 3);
        mark(b, ST_BACKTRANSFORM);
        if (!b->bts.empty()) {
            MmfLaunch Ls = launch_of(b, b->bts, b->d_bts, b->nmax_bts);
            LAUNCH(mmf_launch_backtransform(Ls, b->d_H, b->d_tau, b->d_Vp, b->d_Y, b->d_Zp, fp32), 2);
        }
        if (!b->btc.empty()) {
            MmfLaunch Lc = launch_of(b, b->btc, b->d_btc, b->nmax_btc);
            int nl = 0;
            LAUNCH(mmf_launch_backtransform_tc(Lc, b->btc_n.data(), b->d_H, b->d_tau, b->d_Y, b->d_Zp, b->d_oz,
                                               b->d_btjobs, b->d_status, &nl),
                   0);
            g_launches += nl;
        }
        for (int ci = 0; ci < 4; ++ci) {  // banded systems: Z = Q Y from the chase's reflectors
            if (b->sbt[ci].empty()) continue;
            MmfLaunch Lb = launch_of(b, b->sbt[ci], b->d_sbt[ci], b->nmax_sbt[ci]);
            LAUNCH(mmf_launch_sbr_bt(Lb, 8 << ci, b->d_Zf, b->d_Y, b->d_work, b->d_Zp, fp32), 2);
        }
        if (!b->sbt[4].empty()) {  // the same on the tensor cores (T factors, products, transpose)
            MmfLaunch Lt = launch_of(b, b->sbt[4], b->d_sbt[4], b->nmax_sbt[4]);
            LAUNCH(mmf_launch_sbr_bt_tc(Lt, b->d_Zf, b->d_Y, b->d_work, b->d_oz, (float2*)b->d_Zp, b->d_status), 3);
        }
        if (fp32) LAUNCH(mmf_launch_widen(Ll, b->d_Zp, b->d_Zf, fp32), 1);
    } else {
        mark(b, ST_HETRD);
        mark(b, ST_TRIDIAG);
        mark(b, ST_BACKTRANSFORM);
    }
    mark(b, ST_REFINE);
    if (fp32) {
        MmfLaunch La = launch_of(b, b->all, b->d_all, b->nmax_all);
        LAUNCH(mmf_launch_refine_split_coef(b->d_coef, b->d_coefs, b->n_coef, b->stream), 1);
        LAUNCH(mmf_launch_coef_pattern(La, b->d_coef, b->d_pat), 1);
        LAUNCH(mmf_launch_refine_pre(La, b->d_coefs, b->d_pat, b->d_Zf, b->d_E, b->d_HX, b->d_T, b->d_X1, b->d_oz, b->d_jobs,
                                     b->d_status, 0),
               6);
        mark(b, ST_GRAM);
        // the first step needs G = X^H X only on the band |i - j| <= 16 (far pairs enter its update
        // through C), as the hybrid second step does
        LAUNCH(mmf_launch_refine_band_g(La, b->d_Zf, b->d_R), 1);
        mark(b, ST_REFINE2);
        // every system takes a second step (hybrid or full) below, so the first one applies the
        // near band of Et in FP32
        LAUNCH(mmf_launch_refine_update(La, b->d_coef, b->d_pat, b->d_Zf, b->d_X1, b->d_E, b->d_R, b->d_HX, b->d_T, b->d_E2,
                                        b->d_status, b->d_cid, b->d_oz, b->d_jobs, b->d_Eb, 1, 1),
               9);
        // second step from lam0 = the first step's eigenvalues (E is rewritten at the end)
        CU(cudaMemcpyAsync(b->d_E, b->d_E2, sizeof(double) * b->n_vec, cudaMemcpyDeviceToDevice, b->stream));
        if (!b->rband.empty()) {
            // hybrid: C = X1^H W for all pairs on the tensor cores, G only on the band
            MmfLaunch Lb = launch_of(b, b->rband, b->d_rband, b->nmax_rband);
            LAUNCH(mmf_launch_refine_pre(Lb, b->d_coefs, b->d_pat, b->d_Zf, b->d_E, b->d_HX, b->d_T, b->d_X1, b->d_oz,
                                         b->d_jobs, b->d_status, 2),
                   6);
            LAUNCH(mmf_launch_refine_band_g(Lb, b->d_Zf, b->d_R), 1);
            LAUNCH(mmf_launch_refine_update(Lb, b->d_coef, b->d_pat, b->d_Zf, b->d_X1, b->d_E, b->d_R, b->d_HX, b->d_T,
                                            b->d_E2, b->d_status, b->d_cid, b->d_oz, b->d_jobs, b->d_Eb, 0, 1),
                   9);
        }
        if (!b->rfull.empty()) {
            // full second step: G of the FP64 iterate as G(X1) + C' + C'^H
            MmfLaunch Lf = launch_of(b, b->rfull, b->d_rfull, b->nmax_rfull);
            LAUNCH(mmf_launch_refine_pre(Lf, b->d_coefs, b->d_pat, b->d_Zf, b->d_E, b->d_HX, b->d_T, b->d_X1, b->d_oz,
                                         b->d_jobs, b->d_status, 1),
                   9);
            LAUNCH(refine_gram(b, Lf, 1), 3);
            LAUNCH(mmf_launch_refine_update(Lf, b->d_coef, b->d_pat, b->d_Zf, b->d_X1, b->d_E, b->d_R, b->d_HX, b->d_T,
                                            b->d_E2, b->d_status, b->d_cid, b->d_oz, b->d_jobs, b->d_Eb, 0, 0),
                   9);
        }
        LAUNCH(mmf_launch_refine_finish(La, b->d_Zf, b->d_E, b->d_E2, b->d_S, b->n_mat), 1);
    } else {
        mark(b, ST_GRAM);
        mark(b, ST_REFINE2);
    }
    b->last_stage = 2;
    return MMF_OK;
}

static int stage_outputs(mmf_batch* b) {
    cudaStream_t st = b->stream;
    mark(b, ST_OUTPUTS);
    if (b->n_u > 0) CU(cudaMemsetAsync(b->d_U, 0, sizeof(double2) * b->n_u, st));
    CU(cudaMemsetAsync(b->d_P, 0, sizeof(double) * b->n_p, st));
    MmfLaunch La = launch_of(b, b->all, b->d_all, b->nmax_all);
    // FP32 pieces of Z: the mixed path reuses the refinement's X1 and T buffers (free by now)
    float2* Z1 = b->precision == MMF_MIXED ? b->d_X1 : b->d_Zs;
    float2* Zlo = b->precision == MMF_MIXED ? reinterpret_cast<float2*>(b->d_T) : b->d_Zs + b->n_mat;
    // mixed path: U on the tensor cores (exact slicing) unless a system has too many levels
    // (the int64 sums of the exact slicing bound K = 2M as they bound the Gram product's 2n)
    const bool phi = b->precision == MMF_MIXED && b->nt > 0 && b->Dmax <= mmf_phi_max_levels() &&
                     b->Mmax <= mmf_ozaki_max_n();
    LAUNCH(mmf_launch_outputs(La, b->Mmax, b->Dmax, b->d_E, b->d_Zf, Z1, Zlo, b->d_t, b->t0, b->nt, b->d_F,
                              b->d_U, b->d_P, 1e-8, phi ? 1 : 0, b->d_H,
                              b->precision == MMF_MIXED ? (int)sizeof(float2) : (int)sizeof(double2)),
           b->nt > 0 ? (phi ? 3 : 4) : 1);
    if (phi)
        LAUNCH(mmf_launch_phi(La, b->Dmax, b->nt, Z1, Zlo, b->d_F, b->d_E, b->d_Zf, b->d_t, b->t0, b->d_oz, b->d_U,
                              b->d_status),
               4);
    mark(b, ST_COUNT);
    if (b->timing_runs > 0) b->runs_recorded++;
    b->last_stage = 3;
    return MMF_OK;
}

static int run_stages(mmf_batch* b) {
    int rc = stage_assemble(b);
    if (rc == MMF_OK) rc = stage_eig(b);
    if (rc == MMF_OK) rc = stage_outputs(b);
    return rc;
}

extern "C" int mmf_batch_run(mmf_batch* b) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    if (b->nt > 0 && !b->times_set) return fail(MMF_ERR_STATE, "times not set");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    g_launches = 0;
    if (!b->use_graph) return run_stages(b);
    if (!b->graph_exec) {
        // capture the whole launch sequence once; timing events (if on) record into slot 0
        const int saved = b->runs_recorded;
        b->runs_recorded = 0;
        CU(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        int rc = run_stages(b);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        b->runs_recorded = saved;
        if (rc != MMF_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return fail(MMF_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->graph_exec = nullptr;
            return fail(MMF_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        b->graph_launches = g_launches;
    }
    CU(cudaGraphLaunch(b->graph_exec, b->stream));
    if (b->timing_runs > 0) b->runs_recorded = 1;
    b->last_stage = 3;
    g_launches = b->graph_launches;
    return MMF_OK;
}

extern "C" int mmf_batch_graph(mmf_batch* b, int enable) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    if (b->graph_exec) {
        cudaGraphExecDestroy(b->graph_exec);
        b->graph_exec = nullptr;
    }
    b->use_graph = enable != 0;
    return MMF_OK;
}

extern "C" int mmf_batch_sync(mmf_batch* b, int* status) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    std::vector<int> st(b->count);
    CU(cudaMemcpyAsync(st.data(), b->d_status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    int worst = 0, at = 0;
    for (int i = 0; i < b->count; ++i)
        if (st[i] > worst) worst = st[i], at = i;
    if (status) std::memcpy(status, st.data(), sizeof(int) * b->count);
    // a numeric status replaces the message of any earlier call
    if (worst > 0) return fail(worst, "system " + std::to_string(at) + ": " + mmf_strerror(worst));
    return worst;
}

static int copy_d2h(mmf_batch* b, void* dst, const void* src, size_t bytes) {
    if (!bytes) return MMF_OK;
    CU(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, b->stream));
    return MMF_OK;
}

extern "C" int mmf_batch_get(mmf_batch* b, int i, double* E, double* U, double* P) {
    if (!b || i < 0 || i >= b->count) return fail(MMF_ERR_ARG, "bad batch index");
    if (b->last_stage < 2) return fail(MMF_ERR_STATE, "batch not run");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    const MmfDesc& d = b->desc[i];
    int rc = MMF_OK;
    if (E) rc = copy_d2h(b, E, b->d_E + d.vec_off, sizeof(double) * d.n);
    if (rc == MMF_OK && U) rc = copy_d2h(b, U, b->d_U + d.u_off, sizeof(double2) * (size_t)b->nt * d.D * d.D);
    if (rc == MMF_OK && P) rc = copy_d2h(b, P, b->d_P + d.p_off, sizeof(double) * d.D * d.D);
    if (rc != MMF_OK) return rc;
    CU(cudaStreamSynchronize(b->stream));
    return MMF_OK;
}

extern "C" int mmf_batch_eigenvectors(mmf_batch* b, int i, double* Z) {
    if (!b || i < 0 || i >= b->count || !Z) return fail(MMF_ERR_ARG, "bad batch index or Z");
    if (b->last_stage < 2) return fail(MMF_ERR_STATE, "batch not diagonalised");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    const MmfDesc& d = b->desc[i];
    CU(cudaMemcpy2DAsync(Z, sizeof(double2) * d.n, b->d_Zf + d.mat_off, sizeof(double2) * d.ld,
                         sizeof(double2) * d.n, d.n, cudaMemcpyDeviceToHost, b->stream));
    CU(cudaStreamSynchronize(b->stream));
    return MMF_OK;
}

extern "C" int mmf_batch_results(mmf_batch* b, double* E, double* U, double* P) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    int rc = MMF_OK;
    if (E) rc = copy_d2h(b, E, b->d_E, sizeof(double) * b->n_vec);
    if (rc == MMF_OK && U) rc = copy_d2h(b, U, b->d_U, sizeof(double2) * b->n_u);
    if (rc == MMF_OK && P) rc = copy_d2h(b, P, b->d_P, sizeof(double) * b->n_p);
    if (rc != MMF_OK) return rc;
    CU(cudaStreamSynchronize(b->stream));
    return MMF_OK;
}

extern "C" int64_t mmf_batch_offset(const mmf_batch* b, int what, int i) {
    if (!b || i < 0 || i >= b->count) return -1;
    if (what == 0) return b->desc[i].vec_off;
    if (what == 1) return b->desc[i].u_off;
    if (what == 2) return b->desc[i].p_off;
    return -1;
}

extern "C" int mmf_batch_path(const mmf_batch* b, int i, int* band) {
    if (!b || i < 0 || i >= b->count) return fail(MMF_ERR_ARG, "bad batch index");
    const MmfDesc& d = b->desc[i];
    if (band) *band = d.band;
    if (d.small) return MMF_PATH_JACOBI;
    if (d.band > 0) return MMF_PATH_BAND;
    for (int h : b->huge)
        if (h == i) return MMF_PATH_WHOLE_GPU;
    return MMF_PATH_DENSE;
}

extern "C" int64_t mmf_batch_size(const mmf_batch* b, int what) {
    if (!b) return -1;
    if (what == 0) return b->n_vec;
    if (what == 1) return b->n_u;
    if (what == 2) return b->n_p;
    return -1;
}

// ------------------------------------------------------------------ single-system path
static int solo_ensure(mmf_sys* s, int precision, int nt) {
    if (s->solo && (s->solo->precision != precision || s->solo->nt < nt)) {
        mmf_batch_destroy(s->solo);
        s->solo = nullptr;
    }
    if (!s->solo) {
        mmf_sys* arr[1] = {s};
        int rc = mmf_batch_create(s->ctx, 1, arr, precision, nt, &s->solo);
        if (rc != MMF_OK) return rc;
    }
    return MMF_OK;
}

extern "C" int mmf_build(mmf_sys* s, int precision, int64_t* n_out) {
    if (!s) return fail(MMF_ERR_ARG, "sys is NULL");
    if (s->omega.empty()) return fail(MMF_ERR_ARG, "system has no drive mode");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    int nt = s->solo ? s->solo->nt : 0;
    if (s->solo) { mmf_batch_destroy(s->solo); s->solo = nullptr; }
    int rc = solo_ensure(s, precision, nt);
    if (rc != MMF_OK) return rc;
    CU(cudaSetDevice(s->ctx->device));
    g_launches = 0;
    rc = stage_assemble(s->solo);
    if (rc != MMF_OK) return rc;
    s->state = 1;
    if (n_out) *n_out = s->solo->desc[0].n;
    return MMF_OK;
}

extern "C" int mmf_hamiltonian(mmf_sys* s, double* HF) {
    if (!s || !HF) return fail(MMF_ERR_ARG, "sys and HF required");
    if (s->state != 1 || !s->solo) return fail(MMF_ERR_STATE, "call after mmf_build, before mmf_diagonalise");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    mmf_batch* b = s->solo;
    const MmfDesc& d = b->desc[0];
    CU(cudaSetDevice(s->ctx->device));
    if (b->precision == MMF_FP64) {
        CU(cudaMemcpy2DAsync(HF, sizeof(double2) * d.n, b->d_H, sizeof(double2) * d.ld,
                             sizeof(double2) * d.n, d.n, cudaMemcpyDeviceToHost, s->solo->stream));
        CU(cudaStreamSynchronize(s->solo->stream));
    } else {
        std::vector<float2> tmp((size_t)d.n * d.n);
        CU(cudaMemcpy2DAsync(tmp.data(), sizeof(float2) * d.n, b->d_H, sizeof(float2) * d.ld,
                             sizeof(float2) * d.n, d.n, cudaMemcpyDeviceToHost, s->solo->stream));
        CU(cudaStreamSynchronize(s->solo->stream));
        for (size_t e = 0; e < tmp.size(); ++e) {
            HF[2 * e] = tmp[e].x;
            HF[2 * e + 1] = tmp[e].y;
        }
    }
    return MMF_OK;
}

extern "C" int mmf_diagonalise(mmf_sys* s) {
    if (!s) return fail(MMF_ERR_ARG, "sys is NULL");
    if (s->state < 1 || !s->solo) return fail(MMF_ERR_STATE, "call mmf_build first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    if (s->state >= 2) {  // rebuild: the reduction consumed H_F
        int rc = stage_assemble(s->solo);
        if (rc != MMF_OK) return rc;
    }
    g_launches = 0;
    int rc = stage_eig(s->solo);
    if (rc != MMF_OK) return rc;
    s->state = 2;
    return mmf_batch_sync(s->solo, nullptr);
}

extern "C" int mmf_quasienergies(mmf_sys* s, double* E) {
    if (!s || !E) return fail(MMF_ERR_ARG, "sys and E required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    return mmf_batch_get(s->solo, 0, E, nullptr, nullptr);
}

extern "C" int mmf_eigenvectors(mmf_sys* s, double* Z) {
    if (!s || !Z) return fail(MMF_ERR_ARG, "sys and Z required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    return mmf_batch_eigenvectors(s->solo, 0, Z);
}

// Re-plan the single-system batch for nt times, keeping the eigenpairs on the device.
static int solo_outputs(mmf_sys* s, double t0, int nt, const double* t) {
    mmf_batch* b = s->solo;
    if (b->nt != nt) {
        // a plan with room for nt times; the eigenpairs are recomputed on the new plan
        mmf_batch* nb = nullptr;
        mmf_sys* arr[1] = {s};
        int rc = mmf_batch_create(s->ctx, 1, arr, b->precision, nt, &nb);
        if (rc != MMF_OK) return rc;
        mmf_batch_destroy(b);
        s->solo = b = nb;
        rc = stage_assemble(b);
        if (rc == MMF_OK) rc = stage_eig(b);
        if (rc != MMF_OK) return rc;
    }
    int rc = mmf_batch_set_times(b, t0, t);
    if (rc != MMF_OK) return rc;
    return stage_outputs(b);
}

extern "C" int mmf_time_evolution(mmf_sys* s, double t0, int nt, const double* t, double* U) {
    if (!s || nt < 1 || !t || !U) return fail(MMF_ERR_ARG, "sys, nt >= 1, t and U required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    int rc = solo_outputs(s, t0, nt, t);
    if (rc != MMF_OK) return rc;
    rc = mmf_batch_get(s->solo, 0, nullptr, U, nullptr);
    if (rc != MMF_OK) return rc;
    return mmf_batch_sync(s->solo, nullptr);
}

extern "C" int mmf_transition_avg(mmf_sys* s, double* P) {
    if (!s || !P) return fail(MMF_ERR_ARG, "sys and P required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    mmf_batch* b = s->solo;
    if (b->last_stage < 3) {
        if (b->nt > 0 && !b->times_set) {
            std::vector<double> z((size_t)b->nt, 0.0);
            int rc = mmf_batch_set_times(b, 0.0, z.data());
            if (rc != MMF_OK) return rc;
        }
        int rc = stage_outputs(b);
        if (rc != MMF_OK) return rc;
    }
    return mmf_batch_get(b, 0, nullptr, nullptr, P);
}

extern "C" int mmf_micromotion(mmf_sys* s, int nt, const double* t, double* UF, int64_t* reps) {
    if (!s || nt < 1 || !t || !UF) return fail(MMF_ERR_ARG, "sys, nt >= 1, t and UF required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    mmf_batch* b = s->solo;
    const MmfDesc& d = b->desc[0];
    cudaStream_t st = s->solo->stream;
    const size_t nuf = (size_t)nt * d.D * d.D;
    unsigned char* tmp = nullptr;
    const size_t o_t = 0, o_r = (sizeof(double) * nt + 255) / 256 * 256,
                 o_u = o_r + (sizeof(int64_t) * d.D + 255) / 256 * 256;
    CU(cudaMallocAsync((void**)&tmp, o_u + sizeof(double2) * nuf, st));
    int rc = MMF_OK;
    cudaError_t e = cudaMemcpyAsync(tmp + o_t, t, sizeof(double) * nt, cudaMemcpyHostToDevice, st);
    MmfLaunch L = launch_of(b, b->all, b->d_all, b->nmax_all);
    if (e == cudaSuccess)
        e = mmf_launch_micromotion(L, d.D, b->d_Zf, (const double*)(tmp + o_t), nt, (int64_t*)(tmp + o_r),
                                   (double2*)(tmp + o_u));
    if (e == cudaSuccess) e = cudaMemcpyAsync(UF, tmp + o_u, sizeof(double2) * nuf, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && reps) e = cudaMemcpyAsync(reps, tmp + o_r, sizeof(int64_t) * d.D, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = fail(MMF_ERR_CUDA, std::string("micromotion: ") + cudaGetErrorString(e));
    return rc;
}

extern "C" int mmf_time_evolution_operator(mmf_sys* s, int precision, double t0, int nt,
                                           const double* t, double* U) {
    int64_t n = 0;
    int rc = mmf_build(s, precision, &n);
    if (rc != MMF_OK) return rc;
    rc = mmf_diagonalise(s);
    if (rc < 0) return rc;
    int rc2 = mmf_time_evolution(s, t0, nt, t, U);
    return rc2 != MMF_OK ? rc2 : rc;
}

// ------------------------------------------------------------------ device-pointer variants
// The results go to caller-owned device memory on the caller's stream.  The library's work stays on
// the context stream; the caller's stream waits for it (event), the copy runs on the caller's
// stream, and the context stream then waits for the copy, so later library work cannot overwrite
// the source before it has been read.  Nothing waits on the host.
static int order_after(mmf_ctx* c, cudaStream_t waiter, cudaStream_t producer) {
    if (waiter == producer) return MMF_OK;
    if (!c->order_ev) CU(cudaEventCreateWithFlags(&c->order_ev, cudaEventDisableTiming));
    CU(cudaEventRecord(c->order_ev, producer));
    CU(cudaStreamWaitEvent(waiter, c->order_ev, 0));
    return MMF_OK;
}

// copy `bytes` (rows x width, pitched source) from the library's state to the caller's buffer
static int dev_copy_out(mmf_ctx* c, cudaStream_t lib_st, cudaStream_t user, void* dst, size_t dpitch,
                        const void* src, size_t spitch, size_t width, size_t rows) {
    int rc = order_after(c, user, lib_st);
    if (rc != MMF_OK) return rc;
    if (width && rows) CU(cudaMemcpy2DAsync(dst, dpitch, src, spitch, width, rows, cudaMemcpyDeviceToDevice, user));
    return order_after(c, lib_st, user);
}

extern "C" int mmf_quasienergies_dev(mmf_sys* s, double* E, void* stream) {
    if (!s || !E) return fail(MMF_ERR_ARG, "sys and E required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    mmf_batch* b = s->solo;
    const MmfDesc& d = b->desc[0];
    return dev_copy_out(s->ctx, b->stream, (cudaStream_t)stream, E, sizeof(double) * d.n, b->d_E + d.vec_off,
                        sizeof(double) * d.n, sizeof(double) * d.n, 1);
}

extern "C" int mmf_eigenvectors_dev(mmf_sys* s, double* Z, void* stream) {
    if (!s || !Z) return fail(MMF_ERR_ARG, "sys and Z required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    mmf_batch* b = s->solo;
    const MmfDesc& d = b->desc[0];
    return dev_copy_out(s->ctx, b->stream, (cudaStream_t)stream, Z, sizeof(double2) * d.n, b->d_Zf + d.mat_off,
                        sizeof(double2) * d.ld, sizeof(double2) * d.n, d.n);
}

extern "C" int mmf_time_evolution_dev(mmf_sys* s, double t0, int nt, const double* t, double* U, void* stream) {
    if (!s || nt < 1 || !t || !U) return fail(MMF_ERR_ARG, "sys, nt >= 1, t and U required");
    if (!std::isfinite(t0)) return fail(MMF_ST_NONFINITE, "t0 not finite");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    cudaStream_t user = (cudaStream_t)stream;
    mmf_batch* b = s->solo;
    if (b->nt != nt) {
        // a plan with room for nt times; the eigenpairs are recomputed on the new plan
        mmf_batch* nb = nullptr;
        mmf_sys* arr[1] = {s};
        int rc = mmf_batch_create(s->ctx, 1, arr, b->precision, nt, &nb);
        if (rc != MMF_OK) return rc;
        mmf_batch_destroy(b);
        s->solo = b = nb;
        rc = stage_assemble(b);
        if (rc == MMF_OK) rc = stage_eig(b);
        if (rc != MMF_OK) return rc;
    }
    // the times come from the caller's stream
    int rc = order_after(s->ctx, b->stream, user);
    if (rc != MMF_OK) return rc;
    CU(cudaMemcpyAsync(b->d_t, t, sizeof(double) * nt, cudaMemcpyDeviceToDevice, b->stream));
    b->t0 = t0;
    b->times_set = true;
    rc = stage_outputs(b);
    if (rc != MMF_OK) return rc;
    const MmfDesc& d = b->desc[0];
    const size_t bytes = sizeof(double2) * (size_t)nt * d.D * d.D;
    return dev_copy_out(s->ctx, b->stream, user, U, bytes, b->d_U + d.u_off, bytes, bytes, 1);
}

extern "C" int mmf_transition_avg_dev(mmf_sys* s, double* P, void* stream) {
    if (!s || !P) return fail(MMF_ERR_ARG, "sys and P required");
    if (s->state < 2) return fail(MMF_ERR_STATE, "call mmf_diagonalise first");
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    CU(cudaSetDevice(s->ctx->device));
    mmf_batch* b = s->solo;
    if (b->last_stage < 3) {
        if (b->nt > 0 && !b->times_set) {
            std::vector<double> z((size_t)b->nt, 0.0);
            int rc = mmf_batch_set_times(b, 0.0, z.data());
            if (rc != MMF_OK) return rc;
        }
        int rc = stage_outputs(b);
        if (rc != MMF_OK) return rc;
    }
    const MmfDesc& d = b->desc[0];
    const size_t bytes = sizeof(double) * d.D * d.D;
    return dev_copy_out(s->ctx, b->stream, (cudaStream_t)stream, P, bytes, b->d_P + d.p_off, bytes, bytes, 1);
}

extern "C" int mmf_batch_results_dev(mmf_batch* b, double* E, double* U, double* P, void* stream) {
    if (!b) return fail(MMF_ERR_ARG, "batch is NULL");
    if (b->last_stage < 3) return fail(MMF_ERR_STATE, "batch not run");
    std::lock_guard<std::recursive_mutex> lk(b->ctx->mu);
    CU(cudaSetDevice(b->ctx->device));
    cudaStream_t user = (cudaStream_t)stream;
    int rc = order_after(b->ctx, user, b->stream);
    if (rc != MMF_OK) return rc;
    if (E && b->n_vec) CU(cudaMemcpyAsync(E, b->d_E, sizeof(double) * b->n_vec, cudaMemcpyDeviceToDevice, user));
    if (U && b->n_u) CU(cudaMemcpyAsync(U, b->d_U, sizeof(double2) * b->n_u, cudaMemcpyDeviceToDevice, user));
    if (P && b->n_p) CU(cudaMemcpyAsync(P, b->d_P, sizeof(double) * b->n_p, cudaMemcpyDeviceToDevice, user));
    return order_after(b->ctx, b->stream, user);
}

// ------------------------------------------------------------------ dressed basis (Sec. 3.3, Eq. 4)
extern "C" int mmf_sys_restrict(const mmf_sys* s, int nmodes, const int* modes, mmf_sys** out) {
    if (!out) return fail(MMF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!s || nmodes < 1 || !modes) return fail(MMF_ERR_ARG, "sys, nmodes >= 1 and modes required");
    const int K = (int)s->omega.size();
    for (int k = 0; k < nmodes; ++k) {
        if (modes[k] < 0 || modes[k] >= K) return fail(MMF_ERR_ARG, "mode index out of range");
        for (int q = 0; q < k; ++q)
            if (modes[q] == modes[k]) return fail(MMF_ERR_ARG, "mode listed twice");
    }
    mmf_sys* r = new (std::nothrow) mmf_sys();
    if (!r) return fail(MMF_ERR_NOMEM, "system allocation");
    r->ctx = s->ctx;
    r->D = s->D;
    r->H0 = s->H0;
    for (int k = 0; k < nmodes; ++k) {
        r->omega.push_back(s->omega[modes[k]]);
        r->N.push_back(s->N[modes[k]]);
        r->V.push_back(s->V[modes[k]]);
    }
    *out = r;
    return MMF_OK;
}

extern "C" int64_t mmf_batch_dressed_size(const mmf_batch* b, int what) {
    if (!b) return -1;
    int64_t ne = 0;
    for (const MmfDesc& d : b->desc) ne += d.D;
    if (what == 0) return b->n_u;
    if (what == 1) return ne;
    return -1;
}

extern "C" int64_t mmf_batch_dressed_offset(const mmf_batch* b, int what, int i) {
    if (!b || i < 0 || i >= b->count) return -1;
    if (what == 0) return b->desc[i].u_off;
    if (what == 1) {
        int64_t o = 0;
        for (int q = 0; q < i; ++q) o += b->desc[q].D;
        return o;
    }
    return -1;
}

extern "C" int mmf_batch_dressed(mmf_batch* full, mmf_batch* dress, double* Ud, double* Ebar) {
    if (!full || !dress) return fail(MMF_ERR_ARG, "both batches required");
    if (full->ctx != dress->ctx) return fail(MMF_ERR_ARG, "batches of different contexts");
    if (full->count != dress->count) return fail(MMF_ERR_ARG, "batches of different sizes");
    for (int i = 0; i < full->count; ++i)
        if (full->desc[i].D != dress->desc[i].D) return fail(MMF_ERR_ARG, "system " + std::to_string(i) + ": levels differ");
    if (full->nt < 1) return fail(MMF_ERR_ARG, "the full batch needs times (nt >= 1)");
    if (full->last_stage < 3 || dress->last_stage < 2) return fail(MMF_ERR_STATE, "run both batches first");
    mmf_ctx* c = full->ctx;
    std::lock_guard<std::recursive_mutex> lk(c->mu);
    CU(cudaSetDevice(c->device));
    cudaStream_t st = full->stream;
    int rc = order_after(c, st, dress->stream);
    if (rc != MMF_OK) return rc;
    const int count = full->count, nt = full->nt;
    std::vector<int64_t> roff(count), ufoff(count);
    int64_t ne = 0, nuf = 0;
    int Dmax = 1, nmax_d = 1;
    for (int i = 0; i < count; ++i) {
        const int D = full->desc[i].D;
        roff[i] = ne;
        ufoff[i] = nuf;
        ne += D;
        nuf += (int64_t)(nt + 1) * D * D;
        Dmax = std::max(Dmax, D);
        nmax_d = std::max(nmax_d, dress->desc[i].n);
    }
    // temporaries: offsets, representatives, Ebar, U_F, W, Ud
    Pool p;
    const size_t o_roff = p.take(sizeof(int64_t) * count), o_uoff = p.take(sizeof(int64_t) * count),
                 o_reps = p.take(sizeof(int64_t) * ne), o_eb = p.take(sizeof(double) * ne),
                 o_uf = p.take(sizeof(double2) * nuf), o_w = p.take(sizeof(double2) * full->n_u),
                 o_ud = p.take(sizeof(double2) * full->n_u);
    unsigned char* tmp = nullptr;
    CU(cudaMallocAsync((void**)&tmp, p.off, st));
    cudaError_t e = cudaMemcpyAsync(tmp + o_roff, roff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(tmp + o_uoff, ufoff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = mmf_launch_dressed(dress->d_desc, full->d_desc, count, nmax_d, Dmax, dress->d_Zf, dress->d_E, full->d_U,
                               full->d_t, full->t0, nt, (const int64_t*)(tmp + o_roff), (const int64_t*)(tmp + o_uoff),
                               (int64_t*)(tmp + o_reps), (double*)(tmp + o_eb), (double2*)(tmp + o_uf),
                               (double2*)(tmp + o_w), (double2*)(tmp + o_ud), st);
    if (e == cudaSuccess && Ud)
        e = cudaMemcpyAsync(Ud, tmp + o_ud, sizeof(double2) * full->n_u, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && Ebar) e = cudaMemcpyAsync(Ebar, tmp + o_eb, sizeof(double) * ne, cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(tmp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return fail(MMF_ERR_CUDA, std::string("dressed basis: ") + cudaGetErrorString(e));
    if (st != dress->stream) return order_after(c, dress->stream, st);
    return MMF_OK;
}

extern "C" int mmf_dressed_time_evolution(mmf_sys* s, int ndress, const int* dressing, int precision, double t1,
                                          int nt, const double* t2, double* Ud, double* Ebar) {
    if (!s || nt < 1 || !t2) return fail(MMF_ERR_ARG, "sys, nt >= 1 and t2 required");
    if (s->omega.empty()) return fail(MMF_ERR_ARG, "system has no drive mode");
    mmf_sys* r = nullptr;
    int rc = mmf_sys_restrict(s, ndress, dressing, &r);
    if (rc != MMF_OK) return rc;
    std::lock_guard<std::recursive_mutex> lk(s->ctx->mu);
    mmf_batch *bd = nullptr, *bf = nullptr;
    mmf_sys* a1[1] = {r};
    mmf_sys* a2[1] = {s};
    rc = mmf_batch_create(s->ctx, 1, a1, precision, 0, &bd);
    if (rc == MMF_OK) rc = mmf_batch_run(bd);
    if (rc == MMF_OK) rc = mmf_batch_create(s->ctx, 1, a2, precision, nt, &bf);
    if (rc == MMF_OK) rc = mmf_batch_set_times(bf, t1, t2);
    if (rc == MMF_OK) rc = mmf_batch_run(bf);
    int st1 = 0, st2 = 0;
    if (rc == MMF_OK) st1 = mmf_batch_sync(bd, nullptr);
    if (rc == MMF_OK) st2 = mmf_batch_sync(bf, nullptr);
    if (rc == MMF_OK && (st1 < 0 || st2 < 0)) rc = st1 < 0 ? st1 : st2;
    if (rc == MMF_OK) rc = mmf_batch_dressed(bf, bd, Ud, Ebar);
    if (bf) mmf_batch_destroy(bf);
    if (bd) mmf_batch_destroy(bd);
    mmf_sys_destroy(r);
    if (rc != MMF_OK) return rc;
    return std::max(st1, st2);
}

// ================================================================== serving (continuous batching)
// A worker thread turns queued requests into batch plans on free slots (each slot = one CUDA
// stream with at most one plan in flight), admitting a plan only while the context's HBM budget
// has room for it.  A plan groups requests of the same number of times and the same size class
// (the class of the oldest waiting request first), so a small request never waits for a large
// system's solve.  Plans on different slots overlap on the device; a finished plan's results are
// copied out and the slot takes the next requests at once.  Finished plans stay resident (device
// memory, descriptors, staging) in a small per-server cache keyed by the systems' structure (levels,
// modes, truncations, harmonics) and nt: a later group of the same structure reuses one by uploading
// its own coefficients and times.  Cached plans are released, least recently used first, when a
// new plan needs their memory.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace {
typedef std::chrono::steady_clock Clock;

struct ServeReq {
    uint64_t id = 0;
    mmf_sys* sys = nullptr;  // private copy of the caller's definition
    int nt = 0;
    std::vector<double> t;
    double t0 = 0.0;
    Clock::time_point t_submit, t_done;
    int state = 0;  // 0 queued, 1 on the GPU, 2 done
    int status = 0;
    int64_t n = 0;
    int D = 0;
    int bucket = 0;    // size class of n
    std::string sig;   // structure of the system (what a plan's layout depends on)
    std::vector<double> E, U, P;
};

// size classes of the serving admission: Jacobi-size, small, medium, large
int size_bucket(int64_t n) { return n <= 128 ? 0 : n <= 640 ? 1 : n <= 2500 ? 2 : 3; }

std::string sys_signature(const mmf_sys* s) {
    // the half-bandwidth decides the eigensolver path, so it is part of the layout
    std::string k = std::to_string(s->D) + "b" + std::to_string(sys_band(s));
    for (size_t l = 0; l < s->omega.size(); ++l)
        k += "/" + std::to_string(s->N[l]) + "h" + std::to_string(s->V[l].size());
    return k;
}

struct CachedPlan {
    mmf_batch* b = nullptr;
    std::string sig;
    uint64_t last_use = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    mmf_batch* b = nullptr;
    std::vector<ServeReq*> reqs;
    double* hE = nullptr;
    double2* hU = nullptr;
    double* hP = nullptr;
    int* hst = nullptr;
    size_t capE = 0, capU = 0, capP = 0, capS = 0;
};

template <class T>
int grow_pinned(T** p, size_t* cap, size_t need) {
    if (need <= *cap) return MMF_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    size_t c = std::max(need, *cap * 2);
    cudaError_t e = cudaMallocHost((void**)p, sizeof(T) * c);
    if (e != cudaSuccess) return fail(MMF_ERR_CUDA, std::string("cudaMallocHost: ") + cudaGetErrorString(e));
    *cap = c;
    return MMF_OK;
}
}  // namespace

struct mmf_server {
    mmf_ctx* ctx = nullptr;
    int precision = 0, max_batch = 1;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::thread worker;
    bool stop = false;
    std::deque<ServeReq*> pending;
    std::unordered_map<uint64_t, ServeReq*> reqs;
    uint64_t next_id = 1;
    std::vector<double> lat_ms;
    int64_t completed = 0, solves_started = 0;
    int last_error = 0;
    // resident plans (worker thread only) and the idle stream they are parked on
    std::vector<CachedPlan> cache;
    size_t cache_cap = 8;
    uint64_t use_clock = 0;
    cudaStream_t park = nullptr;
    int64_t plans_created = 0, plans_reused = 0;
};

static std::string plan_signature(const std::vector<ServeReq*>& g) {
    std::string k = std::to_string(g[0]->nt);
    for (const ServeReq* r : g) k += "|" + r->sig;
    return k;
}

// Park a finished plan in the cache (evicting the least recently used beyond the cap).
static void cache_put(mmf_server* sv, mmf_batch* b, const std::string& sig) {
    b->stream = sv->park;  // nothing of it is in flight; later releases wait on an idle stream
    sv->cache.push_back({b, sig, ++sv->use_clock});
    while (sv->cache.size() > sv->cache_cap) {
        auto it = std::min_element(sv->cache.begin(), sv->cache.end(),
                                   [](const CachedPlan& a, const CachedPlan& q) { return a.last_use < q.last_use; });
        mmf_batch_destroy(it->b);
        sv->cache.erase(it);
    }
}

static mmf_batch* cache_take(mmf_server* sv, const std::string& sig) {
    for (auto it = sv->cache.begin(); it != sv->cache.end(); ++it)
        if (it->sig == sig) {
            mmf_batch* b = it->b;
            sv->cache.erase(it);
            return b;
        }
    return nullptr;
}

static bool cache_evict_one(mmf_server* sv) {
    if (sv->cache.empty()) return false;
    auto it = std::min_element(sv->cache.begin(), sv->cache.end(),
                               [](const CachedPlan& a, const CachedPlan& q) { return a.last_use < q.last_use; });
    mmf_batch_destroy(it->b);
    sv->cache.erase(it);
    return true;
}

static mmf_sys* copy_sys(const mmf_sys* s) {
    mmf_sys* c = new (std::nothrow) mmf_sys();
    if (!c) return nullptr;
    c->ctx = s->ctx;
    c->D = s->D;
    c->H0 = s->H0;
    c->omega = s->omega;
    c->N = s->N;
    c->V = s->V;
    return c;
}

// Finish a slot whose plan completed: hand results to the requests, release the plan.
static void serve_finish(mmf_server* sv, Slot& sl) {
    mmf_batch* b = sl.b;
    auto now = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (size_t k = 0; k < sl.reqs.size(); ++k) {
            ServeReq* r = sl.reqs[k];
            const MmfDesc& d = b->desc[k];
            r->E.assign(sl.hE + d.vec_off, sl.hE + d.vec_off + d.n);
            const double* u = (const double*)(sl.hU + d.u_off);
            r->U.assign(u, u + 2 * (size_t)b->nt * d.D * d.D);
            r->P.assign(sl.hP + d.p_off, sl.hP + d.p_off + (size_t)d.D * d.D);
            r->status = sl.hst[k];
            r->t_done = now;
            r->state = 2;
            sv->lat_ms.push_back(std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count());
            sv->completed++;
        }
    }
    cache_put(sv, b, plan_signature(sl.reqs));
    sl.b = nullptr;
    sl.reqs.clear();
    sv->cv.notify_all();
}

// Start a plan for up to max_batch queued requests (same nt and size class as the oldest one) on
// a free slot, reusing a resident plan of the same structure when there is one.  Returns true if
// it started one.
static bool serve_admit(mmf_server* sv, Slot& sl) {
    std::vector<ServeReq*> group;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (sv->pending.empty()) return false;
        const int nt = sv->pending.front()->nt, bucket = sv->pending.front()->bucket;
        for (auto it = sv->pending.begin(); it != sv->pending.end() && (int)group.size() < sv->max_batch; ++it)
            if ((*it)->nt == nt && (*it)->bucket == bucket) group.push_back(*it);
    }
    while (!group.empty()) {
        std::vector<mmf_sys*> sys;
        for (ServeReq* r : group) sys.push_back(r->sys);
        int rc = MMF_OK;
        mmf_batch* b = cache_take(sv, plan_signature(group));
        if (b) {  // same layout: new coefficients into the resident plan
            b->stream = sl.stream;
            b->sys = sys;
            fill_coef(b, b->h_coef);
            for (int i = 0; i < b->count; ++i)  // the frequencies are values, not structure
                for (int k = 0; k < b->desc[i].K; ++k) b->desc[i].omega[k] = sys[i]->omega[k];
            cudaError_t e = cudaMemcpyAsync(b->d_desc, b->desc.data(), sizeof(MmfDesc) * b->count,
                                            cudaMemcpyHostToDevice, sl.stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(b->d_coef, b->h_coef, sizeof(double2) * b->n_coef, cudaMemcpyHostToDevice,
                                    sl.stream);
            if (e != cudaSuccess) rc = fail(MMF_ERR_CUDA, std::string("plan reuse: ") + cudaGetErrorString(e));
            sv->plans_reused++;
        } else {
            rc = batch_create(sv->ctx, (int)sys.size(), sys.data(), sv->precision, group[0]->nt, sl.stream,
                              false, &b);
            if (rc == MMF_ERR_BUDGET) {  // release resident plans, else admit fewer or wait for memory
                if (!cache_evict_one(sv)) group.pop_back();
                continue;
            }
            if (rc == MMF_OK) sv->plans_created++;
        }
        if (rc != MMF_OK) {
            std::lock_guard<std::mutex> lk(sv->mu);
            for (ServeReq* r : group) {
                r->status = rc;
                r->state = 2;
                r->t_done = Clock::now();
                sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
            }
            sv->last_error = rc;
            sv->cv.notify_all();
            return true;
        }
        std::vector<double> t;
        for (ServeReq* r : group) t.insert(t.end(), r->t.begin(), r->t.end());
        rc = mmf_batch_set_times(b, group[0]->t0, t.data());
        if (rc == MMF_OK) rc = mmf_batch_run(b);
        if (rc == MMF_OK) rc = grow_pinned(&sl.hE, &sl.capE, (size_t)std::max<int64_t>(b->n_vec, 1));
        if (rc == MMF_OK) rc = grow_pinned(&sl.hU, &sl.capU, (size_t)std::max<int64_t>(b->n_u, 1));
        if (rc == MMF_OK) rc = grow_pinned(&sl.hP, &sl.capP, (size_t)std::max<int64_t>(b->n_p, 1));
        if (rc == MMF_OK) rc = grow_pinned(&sl.hst, &sl.capS, (size_t)b->count);
        cudaError_t e = cudaSuccess;
        if (rc == MMF_OK) e = cudaMemcpyAsync(sl.hE, b->d_E, sizeof(double) * b->n_vec, cudaMemcpyDeviceToHost, sl.stream);
        if (rc == MMF_OK && e == cudaSuccess && b->n_u > 0)
            e = cudaMemcpyAsync(sl.hU, b->d_U, sizeof(double2) * b->n_u, cudaMemcpyDeviceToHost, sl.stream);
        if (rc == MMF_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(sl.hP, b->d_P, sizeof(double) * b->n_p, cudaMemcpyDeviceToHost, sl.stream);
        if (rc == MMF_OK && e == cudaSuccess)
            e = cudaMemcpyAsync(sl.hst, b->d_status, sizeof(int) * b->count, cudaMemcpyDeviceToHost, sl.stream);
        if (rc == MMF_OK && e == cudaSuccess) e = cudaEventRecord(sl.done, sl.stream);
        if (rc == MMF_OK && e != cudaSuccess) rc = fail(MMF_ERR_CUDA, cudaGetErrorString(e));
        std::lock_guard<std::mutex> lk(sv->mu);
        for (ServeReq* r : group) sv->pending.erase(std::find(sv->pending.begin(), sv->pending.end(), r));
        if (rc != MMF_OK) {
            for (ServeReq* r : group) {
                r->status = rc;
                r->state = 2;
                r->t_done = Clock::now();
            }
            sv->last_error = rc;
            mmf_batch_destroy(b);
            sv->cv.notify_all();
            return true;
        }
        for (ServeReq* r : group) r->state = 1;
        sl.b = b;
        sl.reqs = group;
        sv->solves_started += (int64_t)group.size();
        return true;
    }
    return false;  // not even one request fits the budget right now
}

static void serve_loop(mmf_server* sv) {
    cudaSetDevice(sv->ctx->device);
    while (true) {
        bool progress = false;
        for (Slot& sl : sv->slots)
            if (sl.b && cudaEventQuery(sl.done) == cudaSuccess) {
                serve_finish(sv, sl);
                progress = true;
            }
        for (Slot& sl : sv->slots)
            if (!sl.b && serve_admit(sv, sl)) progress = true;
        std::unique_lock<std::mutex> lk(sv->mu);
        if (sv->stop) {
            bool busy = false;
            for (Slot& sl : sv->slots) busy |= sl.b != nullptr;
            if (!busy) break;
        }
        if (!progress) sv->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

extern "C" int mmf_serve_create(mmf_ctx* ctx, int slots, int max_batch, int precision, mmf_server** out) {
    if (!out) return fail(MMF_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ctx || slots < 1 || slots > 64 || max_batch < 1) return fail(MMF_ERR_ARG, "bad server arguments");
    if (precision != MMF_FP64 && precision != MMF_MIXED) return fail(MMF_ERR_ARG, "bad precision");
    CU(cudaSetDevice(ctx->device));
    mmf_server* sv = new (std::nothrow) mmf_server();
    if (!sv) return fail(MMF_ERR_NOMEM, "server allocation");
    sv->ctx = ctx;
    sv->precision = precision;
    sv->max_batch = max_batch;
    sv->slots.resize(slots);
    sv->cache_cap = (size_t)std::max(4, 2 * slots);
    if (cudaStreamCreateWithFlags(&sv->park, cudaStreamNonBlocking) != cudaSuccess) {
        delete sv;
        return fail(MMF_ERR_CUDA, "server stream");
    }
    for (Slot& sl : sv->slots) {
        cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (Slot& q : sv->slots) {
                if (q.stream) cudaStreamDestroy(q.stream);
                if (q.done) cudaEventDestroy(q.done);
            }
            cudaStreamDestroy(sv->park);
            delete sv;
            return fail(MMF_ERR_CUDA, cudaGetErrorString(e));
        }
    }
    sv->worker = std::thread(serve_loop, sv);
    *out = sv;
    return MMF_OK;
}

extern "C" int mmf_serve_submit(mmf_server* sv, const mmf_sys* sys, int nt, const double* t, double t0,
                                uint64_t* ticket) {
    if (!sv || !sys || nt < 0 || (nt > 0 && !t) || !ticket) return fail(MMF_ERR_ARG, "bad submit arguments");
    if (sys->ctx != sv->ctx) return fail(MMF_ERR_ARG, "system from another context");
    if (sys->omega.empty()) return fail(MMF_ERR_ARG, "system has no drive mode");
    ServeReq* r = new (std::nothrow) ServeReq();
    if (!r) return fail(MMF_ERR_NOMEM, "request allocation");
    r->sys = copy_sys(sys);
    if (!r->sys) { delete r; return fail(MMF_ERR_NOMEM, "request allocation"); }
    r->nt = nt;
    r->t.assign(t, t + nt);
    r->t0 = t0;
    r->n = sys_dim(sys);
    r->D = sys->D;
    r->bucket = size_bucket(r->n);
    r->sig = sys_signature(sys);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        r->id = sv->next_id++;
        sv->pending.push_back(r);
        sv->reqs[r->id] = r;
        *ticket = r->id;
    }
    sv->cv.notify_all();
    return MMF_OK;
}

extern "C" int mmf_serve_poll(mmf_server* sv, uint64_t ticket, int* done) {
    if (!sv || !done) return fail(MMF_ERR_ARG, "bad poll arguments");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(MMF_ERR_ARG, "unknown ticket");
    *done = it->second->state == 2;
    return MMF_OK;
}

extern "C" int mmf_serve_wait(mmf_server* sv, uint64_t ticket, int timeout_ms, double* E, double* U, double* P,
                              int* status) {
    if (!sv) return fail(MMF_ERR_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end()) return fail(MMF_ERR_ARG, "unknown ticket");
    ServeReq* r = it->second;
    auto ready = [&] { return r->state == 2; };
    if (timeout_ms < 0) sv->cv.wait(lk, ready);
    else if (!sv->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(MMF_ERR_STATE, "request not finished within the timeout");
    if (status) *status = r->status;
    if (r->status < 0) {
        sv->reqs.erase(it);
        mmf_sys_destroy(r->sys);
        delete r;
        return fail(MMF_ERR_CUDA, "request failed");
    }
    if (E) std::memcpy(E, r->E.data(), sizeof(double) * r->E.size());
    if (U) std::memcpy(U, r->U.data(), sizeof(double) * r->U.size());
    if (P) std::memcpy(P, r->P.data(), sizeof(double) * r->P.size());
    sv->reqs.erase(it);
    mmf_sys_destroy(r->sys);
    delete r;
    return MMF_OK;
}

extern "C" int mmf_serve_stats(mmf_server* sv, double* p50_ms, double* p99_ms, double* mean_ms,
                               int64_t* completed) {
    if (!sv) return fail(MMF_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::vector<double> v = sv->lat_ms;
    std::sort(v.begin(), v.end());
    auto q = [&](double f) { return v.empty() ? 0.0 : v[std::min(v.size() - 1, (size_t)(f * (v.size() - 1) + 0.5))]; };
    double m = 0.0;
    for (double x : v) m += x;
    if (p50_ms) *p50_ms = q(0.50);
    if (p99_ms) *p99_ms = q(0.99);
    if (mean_ms) *mean_ms = v.empty() ? 0.0 : m / v.size();
    if (completed) *completed = sv->completed;
    return MMF_OK;
}

extern "C" int mmf_serve_plan_stats(mmf_server* sv, int64_t* created, int64_t* reused, int64_t* resident) {
    if (!sv) return fail(MMF_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (created) *created = sv->plans_created;
    if (reused) *reused = sv->plans_reused;
    if (resident) *resident = (int64_t)sv->cache.size();
    return MMF_OK;
}

extern "C" int mmf_serve_reset_stats(mmf_server* sv) {
    if (!sv) return fail(MMF_ERR_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat_ms.clear();
    sv->completed = 0;
    return MMF_OK;
}

extern "C" int mmf_serve_destroy(mmf_server* sv) {
    if (!sv) return MMF_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
        for (ServeReq* r : sv->pending) {  // never started
            r->status = MMF_ERR_STATE;
            r->state = 2;
        }
        sv->pending.clear();
    }
    sv->cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    for (auto& kv : sv->reqs) {
        mmf_sys_destroy(kv.second->sys);
        delete kv.second;
    }
    for (CachedPlan& cp : sv->cache) mmf_batch_destroy(cp.b);
    sv->cache.clear();
    if (sv->park) cudaStreamDestroy(sv->park);
    for (Slot& sl : sv->slots) {
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        if (sl.hE) cudaFreeHost(sl.hE);
        if (sl.hU) cudaFreeHost(sl.hU);
        if (sl.hP) cudaFreeHost(sl.hP);
        if (sl.hst) cudaFreeHost(sl.hst);
    }
    delete sv;
    return MMF_OK;
}

// ================================================================== diagnostics
extern "C" int mmf_selftest_tensor_cores(int M, int N, int K, int kind, int products, double* max_abs_err,
                                         double* max_abs_ref) {
    if (!max_abs_err || !max_abs_ref) return fail(MMF_ERR_ARG, "output pointers required");
    int rc = mmf_umma_selftest_impl(M, N, K, kind, products, max_abs_err, max_abs_ref);
    if (rc == -1) return fail(MMF_ERR_ARG, "bad self-test sizes");
    if (rc == -4) return fail(MMF_ERR_CUDA, "self-test CUDA failure");
    if (rc == 1) return fail(MMF_ST_NOCONV, "tensor-core pipeline wait timed out");
    return MMF_OK;
}

extern "C" int mmf_selftest_split_tf32(int M, int N, int K, int mode, double* max_rel_err,
                                       double* max_rel_err_fp32) {
    if (!max_rel_err || !max_rel_err_fp32) return fail(MMF_ERR_ARG, "output pointers required");
    int rc = mmf_tf3_selftest_impl(M, N, K, mode, max_rel_err, max_rel_err_fp32);
    if (rc == -1) return fail(MMF_ERR_ARG, "bad self-test sizes or mode");
    if (rc == -4) return fail(MMF_ERR_CUDA, "self-test CUDA failure");
    if (rc == 1) return fail(MMF_ST_NOCONV, "tensor-core pipeline wait timed out");
    return MMF_OK;
}

extern "C" int mmf_selftest_hetrd(int n, int count, int tensor_cores, double* max_abs_err, double* max_abs_ref) {
    if (!max_abs_err || !max_abs_ref) return fail(MMF_ERR_ARG, "output pointers required");
    int rc = mmf_hetrd_selftest_impl(n, count, tensor_cores, max_abs_err, max_abs_ref);
    if (rc == -1) return fail(MMF_ERR_ARG, "bad self-test sizes");
    if (rc == -4) return fail(MMF_ERR_CUDA, "self-test CUDA failure");
    if (rc == 1) return fail(MMF_ST_NOCONV, "tensor-core pipeline wait timed out");
    return MMF_OK;
}

extern "C" int mmf_selftest_gram(int n, double* max_abs_err, double* max_abs_ref) {
    if (!max_abs_err || !max_abs_ref) return fail(MMF_ERR_ARG, "output pointers required");
    int rc = mmf_ozaki_selftest_impl(n, max_abs_err, max_abs_ref);
    if (rc == -1) return fail(MMF_ERR_ARG, "bad self-test size");
    if (rc == -4) return fail(MMF_ERR_CUDA, "self-test CUDA failure");
    if (rc == 1) return fail(MMF_ST_NOCONV, "tensor-core pipeline wait timed out");
    return MMF_OK;
}
