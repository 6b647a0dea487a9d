// k_ozaki.cu -- the refinement's Gram matrix G = X1^H X1 (X1 FP32-exact) on the BF16 tensor
// cores, FP64-accurate, by exact integer slicing (the error-free splitting of Ozaki, Ogita, Oishi
// & Rump, Numer. Algorithms 59 (2012)).
//
// Real form: with a_i = [Re x_i | Im x_i] and a'_j = [Im x_j | -Re x_j] (x_i column i of X1,
// K = 2n), Re G_ij = a_i . a_j and Im G_ij = a_i . a'_j.
//
// Slicing (k_oz_slice): column i is scaled by 2^-e_i (e_i the exponent of its largest entry, so
// every scaled entry t lies in (-1, 1)) and cut into OZ_S integer slices of OZ_W bits,
//     t = sum_s 2^-OZ_W(s+1) v_s,   v_0 in [-64, 64], v_s in [-32, 32] (s > 0),
// each step t <- 64 t - rint(64 t) exact in FP32; the integers are exact in BF16.  The slices
// cover 42 bits below each column's largest entry.
//
// Products (k_oz_gram): for every slice pair (a, b) with a + b <= OZ_L, S_a S_b^T is an integer
// matrix.  On the tensor cores, BF16 products of these integers are exact and so is their FP32
// accumulation as long as every partial sum stays below 2^24: K is taken in chunks of OZ_KCH
// (<= 3968 terms of magnitude <= 2^12), and after each chunk the FP32 accumulator (an exact
// integer) is added into an int64 accumulator per output, scaled by 2^(6 (OZ_L - a - b) - 6)
// (the pairs with a + b = OZ_L lose their 6 lowest bits, 2^-42 of the leading term).  At the
// end G_ij = 2^(e_i + e_j - 6 (OZ_L + 2) + 6) acc_ij, one rounding to FP64.
// Error: the dropped pairs and slice remainders are below ~2^-40 |x_i| |x_j| per entry.
//
// One CTA of 128 threads per 128 x 64 tile of the lower triangle (Re and Im accumulated side by
// side in TMEM: columns 0..63 and 64..127), two cp.async stages of A (128 rows) and B, B' (64 rows)
// in the 128-byte-swizzled K-major layout, one thread issuing tcgen05.mma, int64 accumulators in
// shared memory [column][row].  Every mbarrier wait is bounded; a time-out sets *err, frees
// TMEM and leaves.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "mmf_internal.h"
#include "umma_common.h"

#define OZ_W 6
#define OZ_L 6                 // pairs a + b <= OZ_L
#define OZ_THREADS 128
#define OZ_TM 128
#define OZ_TN 64
#define OZ_KSTEP 64            // BF16 elements of K per stage (one 128-byte row segment)
#define OZ_KCH (62 * OZ_KSTEP) // K per exact FP32 accumulation: 3968 * 2^12 < 2^24
#define OZ_STAGE_BYTES (16384 + 8192 + 8192)

static_assert(OZ_S == OZ_L + 1, "slices cover the kept pairs");

__host__ __device__ __forceinline__ int oz_la(int n) { return (2 * n + OZ_KSTEP - 1) / OZ_KSTEP * OZ_KSTEP; }

// ------------------------------------------------------------------ slicing
// One warp per column: scale exponent, then the OZ_S slices of a_i (Sa) and a'_i (Sb).
// Slice s of system d: Sa + oz_off + s * n * la (rows i, la BF16 each); Sb likewise after the
// OZ_S Sa slices.
__global__ void __launch_bounds__(256) k_oz_slice(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                  const float2* __restrict__ X1g, __nv_bfloat16* __restrict__ S,
                                                  int* __restrict__ expg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = oz_la(n);
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= n) return;
    const float2* x = X1g + d.mat_off + (int64_t)i * d.ld;
    float m = 0.f;
    for (int k = lane; k < n; k += 32) m = fmaxf(m, fmaxf(fabsf(x[k].x), fabsf(x[k].y)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.f) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1): |x| 2^-e < 1
    if (lane == 0) expg[d.vec_off + i] = e;
    const int64_t plane = (int64_t)n * la;
    __nv_bfloat16* Sa = S + d.oz_off + (int64_t)i * la;
    __nv_bfloat16* Sb = Sa + OZ_S * plane;
    for (int k = lane; k < la; k += 32) {
        float tr = 0.f, ti = 0.f;  // the two entries of a_i that k and k + n address
        if (k < n) {
            tr = ldexpf(x[k].x, -e);  // a_i[k] = Re x_ki; a'_i[k + n] = -Re x_ki
            ti = ldexpf(x[k].y, -e);  // a_i[k + n] = Im x_ki; a'_i[k] = Im x_ki
        }
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            tr *= 64.f;
            ti *= 64.f;
            const float vr = rintf(tr), vi = rintf(ti);
            tr -= vr;
            ti -= vi;
            if (k < n) {
                Sa[s * plane + k] = __float2bfloat16_rn(vr);
                Sa[s * plane + n + k] = __float2bfloat16_rn(vi);
                Sb[s * plane + k] = __float2bfloat16_rn(vi);
                Sb[s * plane + n + k] = __float2bfloat16_rn(-vr);
            } else if (k >= 2 * n) {  // row padding
                Sa[s * plane + k] = __float2bfloat16_rn(0.f);
                Sb[s * plane + k] = __float2bfloat16_rn(0.f);
            }
        }
    }
}

// ------------------------------------------------------------------ products
__device__ __forceinline__ void oz_load(uint32_t sbase, const __nv_bfloat16* g, int rows, int rows_valid,
                                        int64_t k0, int la) {
    // rows x 128 bytes, 16-byte chunks into the swizzled K-major layout
    for (int c = threadIdx.x; c < rows * 8; c += OZ_THREADS) {
        const int r = c >> 3, j = c & 7;
        const uint32_t dst = sbase + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
        const bool ok = r < rows_valid;
        const void* src = ok ? (const void*)(g + (int64_t)r * la + k0 + j * 8) : (const void*)g;
        cp_async16(dst, src, ok ? 16 : 0);
    }
}

// tile t of the lower triangle of an n x n matrix in OZ_TM x OZ_TN tiles: (I, J) with J <= 2 I + 1
__device__ __forceinline__ bool oz_tile(int t, int n, int& I, int& J) {
    const int nI = (n + OZ_TM - 1) / OZ_TM, nJ = (n + OZ_TN - 1) / OZ_TN;
    for (I = 0; I < nI; ++I) {
        const int cnt = min(2 * I + 2, nJ);
        if (t < cnt) {
            J = t;
            return true;
        }
        t -= cnt;
    }
    return false;
}

__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_gram(const MmfDesc* __restrict__ descs,
                                                           const int* __restrict__ idx,
                                                           const __nv_bfloat16* __restrict__ S,
                                                           const int* __restrict__ expg, double2* __restrict__ Gg,
                                                           int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ uint64_t bar[2];
    __shared__ uint32_t tmem_s;
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = oz_la(n);
    int I, J;
    if (!oz_tile(blockIdx.x, n, I, J)) return;
    const int i0 = I * OZ_TM, j0 = J * OZ_TN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    long long* acc = reinterpret_cast<long long*>(base + 2 * OZ_STAGE_BYTES);  // [2][OZ_TN][OZ_TM]
    for (int e = threadIdx.x; e < 2 * OZ_TN * OZ_TM; e += OZ_THREADS) acc[e] = 0;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const uint32_t idesc = umma_idesc_mn(1, OZ_TM, OZ_TN);
    const int64_t plane = (int64_t)n * la;
    const __nv_bfloat16* Sys = S + d.oz_off;
    uint32_t phase[2] = {0u, 0u};  // parity of the next phase to wait for, per stage barrier
    bool ok = true;

    for (int a = 0; a <= OZ_L && ok; ++a) {
        for (int b = 0; a + b <= OZ_L && ok; ++b) {
            const __nv_bfloat16* Ag = Sys + a * plane + (int64_t)i0 * la;
            const __nv_bfloat16* Bg = Sys + b * plane + (int64_t)j0 * la;
            const __nv_bfloat16* Bpg = Sys + (OZ_S + b) * plane + (int64_t)j0 * la;
            const int sh = 6 * (OZ_L - a - b) - 6;
            for (int kc0 = 0; kc0 < la && ok; kc0 += OZ_KCH) {
                const int nk = (min(la, kc0 + OZ_KCH) - kc0) / OZ_KSTEP;
                // stage 0 of the chunk (every earlier MMA has completed: both stages are free)
                {
                    const uint32_t st = sbase;
                    oz_load(st, Ag, OZ_TM, n - i0, kc0, la);
                    oz_load(st + 16384, Bg, OZ_TN, n - j0, kc0, la);
                    oz_load(st + 24576, Bpg, OZ_TN, n - j0, kc0, la);
                    asm volatile("cp.async.commit_group;" ::: "memory");
                }
                for (int kk = 0; kk < nk && ok; ++kk) {
                    const int s = kk & 1;
                    if (kk + 1 < nk) {
                        const int s1 = s ^ 1;
                        if (kk >= 1) {  // the MMAs of step kk-1 read stage s1: wait for their commit
                            ok = __syncthreads_and(mbar_wait(&bar[s1], phase[s1]) ? 1 : 0) != 0;
                            phase[s1] ^= 1u;
                            if (!ok) break;
                        }
                        const uint32_t st = sbase + s1 * OZ_STAGE_BYTES;
                        const int64_t k1 = kc0 + (int64_t)(kk + 1) * OZ_KSTEP;
                        oz_load(st, Ag, OZ_TM, n - i0, k1, la);
                        oz_load(st + 16384, Bg, OZ_TN, n - j0, k1, la);
                        oz_load(st + 24576, Bpg, OZ_TN, n - j0, k1, la);
                        asm volatile("cp.async.commit_group;" ::: "memory");
                        asm volatile("cp.async.wait_group 1;" ::: "memory");
                    } else {
                        asm volatile("cp.async.wait_group 0;" ::: "memory");
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t st = sbase + s * OZ_STAGE_BYTES;
                        const uint64_t da = umma_desc(st), db = umma_desc(st + 16384), dbp = umma_desc(st + 24576);
#pragma unroll
                        for (int q = 0; q < OZ_KSTEP / 16; ++q) {  // 32 bytes of K per instruction
                            const uint32_t accf = (kk > 0 || q > 0) ? 1u : 0u;
                            const uint64_t adv = (uint64_t)((q * 32) >> 4);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                                "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(accf)
                                : "memory");
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + OZ_TN),
                                "l"(da + adv), "l"(dbp + adv), "r"(idesc), "r"(accf)
                                : "memory");
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                smem_u32(&bar[s]))
                            : "memory");
                    }
                }
                if (!ok) break;
                // wait for the chunk's last commit, then drain TMEM into the int64 accumulators
                {
                    const int s = (nk - 1) & 1;
                    ok = __syncthreads_and(mbar_wait(&bar[s], phase[s]) ? 1 : 0) != 0;
                    phase[s] ^= 1u;
                    // the other stage's commit (if any) precedes this one and is complete too
                    if (ok && nk >= 2) {
                        const int s1 = s ^ 1;
                        ok = __syncthreads_and(mbar_wait(&bar[s1], phase[s1]) ? 1 : 0) != 0;
                        phase[s1] ^= 1u;
                    }
                }
                if (!ok) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const int row = warp * 32 + lane;
#pragma unroll 1
                for (int c0 = 0; c0 < 2 * OZ_TN; c0 += 32) {
                    uint32_t v[32];
                    const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
                          "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]),
                          "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]),
                          "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]),
                          "=r"(v[31])
                        : "r"(ta));
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const long long iv = __float2ll_rn(__uint_as_float(v[q]));  // an exact integer
                        const long long term = sh >= 0 ? (iv << sh) : (iv >> (-sh));
                        acc[(int64_t)(c0 + q) * OZ_TM + row] += term;
                    }
                }
                // TMEM is overwritten by the next chunk's first MMA only after every thread's loads
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
            }
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (ok) {
        __syncthreads();
        const int row = warp * 32 + lane;
        const int i = i0 + row;
        if (i < n) {
            const int ei = expg[d.vec_off + i];
            double2* G = Gg + d.mat_off;
            for (int c = 0; c < OZ_TN; ++c) {
                const int j = j0 + c;
                if (j >= n || j > i) continue;
                const int sc = ei + expg[d.vec_off + j] - 6 * (OZ_L + 2) + 6;
                const double gr = ldexp((double)acc[(int64_t)c * OZ_TM + row], sc);
                const double gi = (i == j) ? 0.0 : ldexp((double)acc[(int64_t)(OZ_TN + c) * OZ_TM + row], sc);
                G[(int64_t)j * d.ld + i] = make_double2(gr, gi);
                if (i != j) G[(int64_t)i * d.ld + j] = make_double2(gr, -gi);
            }
        }
    } else if (threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128u) : "memory");
}

size_t mmf_ozaki_slice_elems(int n) { return (size_t)2 * OZ_S * n * oz_la(n); }

cudaError_t mmf_launch_ozaki_gram(const MmfLaunch& L, const float2* X1, void* S, int* exps, double2* G, int* err) {
    if (L.count <= 0) return cudaSuccess;
    k_oz_slice<<<dim3((L.nmax + 7) / 8, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X1, (__nv_bfloat16*)S, exps);
    const int nI = (L.nmax + OZ_TM - 1) / OZ_TM, nJ = (L.nmax + OZ_TN - 1) / OZ_TN;
    int tiles = 0;
    for (int I = 0; I < nI; ++I) tiles += std::min(2 * I + 2, nJ);
    const size_t sm = 2 * (size_t)OZ_STAGE_BYTES + sizeof(long long) * 2 * OZ_TN * OZ_TM + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_oz_gram<<<dim3(tiles, L.count), OZ_THREADS, sm, L.stream>>>(L.desc, L.idx, (const __nv_bfloat16*)S, exps, G,
                                                                   err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ self-test
// G of one seeded n x n FP32 matrix (columns of unit norm, entries spread over several orders
// of magnitude) against an FP64 reference; returns the largest |G - G_ref|.
__global__ void k_oz_fill(float2* X, int n, int ld, uint32_t seed) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * ld;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(e / ld), r = (int)(e % ld);
        uint32_t h = (uint32_t)e * 2654435761u ^ seed;
        h ^= h >> 13; h *= 0x5bd1e995u; h ^= h >> 15;
        const float u = ((h & 0xFFFF) + 0.5f) / 65536.f - 0.5f, v = (((h >> 16) & 0xFFFF) + 0.5f) / 65536.f - 0.5f;
        const float mag = exp2f(-(float)((h >> 8) % 20));  // 2^0 .. 2^-19
        X[e] = r < n ? make_float2(u * mag, v * mag) : make_float2(0.f, 0.f);
        (void)c;
    }
}
__global__ void k_oz_ref(const float2* X, int n, int ld, double2* R) {
    const int i = blockIdx.y, j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || i >= n) return;
    double re = 0.0, im = 0.0;
    for (int k = 0; k < n; ++k) {
        const float2 a = X[(int64_t)i * ld + k], b = X[(int64_t)j * ld + k];
        re += (double)a.x * b.x + (double)a.y * b.y;  // conj(a) b, products exact in FP64
        im += (double)a.x * b.y - (double)a.y * b.x;
    }
    R[(int64_t)j * ld + i] = make_double2(re, im);
}
__global__ void k_oz_cmp(const double2* G, const double2* R, int n, int ld, double* out) {
    double mx = 0.0, ref = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)n * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), i = (int)(e % n);
        const double2 g = G[(int64_t)j * ld + i], r = R[(int64_t)j * ld + i];
        mx = fmax(mx, fmax(fabs(g.x - r.x), fabs(g.y - r.y)));
        ref = fmax(ref, fmax(fabs(r.x), fabs(r.y)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        ref = fmax(ref, __shfl_xor_sync(0xffffffffu, ref, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long*)&out[0], __double_as_longlong(mx));
        atomicMax((unsigned long long*)&out[1], __double_as_longlong(ref));
    }
}

int mmf_ozaki_selftest_impl(int n, double* max_abs, double* max_ref) {
    if (n < 1 || n > 8192) return -1;
    const int ld = (n + 3) / 4 * 4;
    MmfDesc hd;
    memset(&hd, 0, sizeof(hd));
    hd.n = n; hd.ld = ld; hd.D = 1; hd.M = n;
    float2* X = nullptr;
    double2 *G = nullptr, *R = nullptr;
    double* out = nullptr;
    void* S = nullptr;
    int *ex = nullptr, *err = nullptr, *didx = nullptr;
    MmfDesc* dd = nullptr;
    int rc = 0;
    cudaError_t e = cudaMalloc(&X, sizeof(float2) * (size_t)n * ld);
    if (e == cudaSuccess) e = cudaMalloc(&G, sizeof(double2) * (size_t)n * ld);
    if (e == cudaSuccess) e = cudaMalloc(&R, sizeof(double2) * (size_t)n * ld);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(uint16_t) * mmf_ozaki_slice_elems(n));
    if (e == cudaSuccess) e = cudaMalloc(&ex, sizeof(int) * n);
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&didx, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&dd, sizeof(MmfDesc));
    if (e == cudaSuccess) e = cudaMemset(out, 0, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(didx, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(G, 0, sizeof(double2) * (size_t)n * ld);
    if (e == cudaSuccess) e = cudaMemcpy(dd, &hd, sizeof(hd), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_oz_fill<<<256, 256>>>(X, n, ld, 4242u);
        MmfLaunch L;
        L.desc = dd; L.idx = didx; L.count = 1; L.nmax = n; L.stream = 0;
        e = mmf_launch_ozaki_gram(L, X, S, ex, G, err);
    }
    if (e == cudaSuccess) {
        k_oz_ref<<<dim3((n + 127) / 128, n), 128>>>(X, n, ld, R);
        k_oz_cmp<<<256, 256>>>(G, R, n, ld, out);
        e = cudaDeviceSynchronize();
    }
    double hout[2] = {0, 0};
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(hout, out, sizeof(hout), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = -4;
    else if (herr) rc = 1;
    *max_abs = hout[0];
    *max_ref = hout[1];
    cudaFree(X); cudaFree(G); cudaFree(R); cudaFree(out); cudaFree(S); cudaFree(ex); cudaFree(err);
    cudaFree(didx); cudaFree(dd);
    return rc;
}
