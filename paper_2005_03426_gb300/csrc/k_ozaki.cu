// k_ozaki.cu -- the refinement's Gram matrix G = X1^H X1 (X1 FP32-exact) on the BF16 tensor
// cores, FP64-accurate, by exact integer slicing (the error-free splitting of Ozaki, Ogita, Oishi
// & Rump, Numer. Algorithms 59 (2012)).
//
// Real form: with a_i = [Re x_i | Im x_i] and a'_j = [Im x_j | -Re x_j] (x_i column i of X1,
// K = 2n), Re G_ij = a_i . a_j and Im G_ij = a_i . a'_j.
//
// Slicing (k_oz_slice): column i is scaled by 2^-(e_i + 1) (e_i the exponent of its largest
// entry, so every scaled entry t lies in (-1/2, 1/2)) and cut into OZ_S integer slices of OZ_W
// bits,
//     t = sum_s 2^-OZ_W(s+1) v_s,   v_s in [-128, 128],
// each step t <- 256 t - rint(256 t) exact in FP32; the integers are exact in BF16 (which holds
// integers up to 256).  The slices cover 40 bits below each column's largest entry.
//
// Products (k_oz_gram): for every slice pair (a, b) with a + b <= OZ_L, S_a S_b^T is an integer
// matrix.  On the tensor cores, BF16 products of these integers are exact and so is their FP32
// accumulation as long as every partial sum stays within 2^24: K is taken in chunks of OZ_KCH
// (1024 terms of magnitude <= 2^14), and after each chunk the FP32 accumulator (an exact
// integer) is added into an int64 accumulator per output, scaled by 2^(OZ_W (OZ_L - a - b)).  At
// the end G_ij = 2^(e_i + e_j + 2 - OZ_W (OZ_L + 2)) acc_ij, one rounding to FP64.  The int64
// sums stay below 2^63 for 2n <= 2^17 (n <= OZ_NMAX).
// Error: the dropped pairs and slice remainders are below ~2^-38 |x_i| |x_j| per entry.
//
// Data layout: the slicing kernel writes every slice pre-tiled in the shared-memory layout the
// tensor cores read (64-row x 64-K tiles of 8 KB, 128-byte swizzle, K-major), so one stage of
// operands is three bulk copies.  One CTA per 128 x 64 tile of the lower triangle of G, six warps:
//   warp 4 (one lane): producer, fills a ring of OZ_STAGES stages (A 16 KB, B 8 KB, B' 8 KB) with
//                      cp.async.bulk, completion counted on full[stage];
//   warp 5 (one lane): MMA issuer, tcgen05.mma into one of two TMEM accumulators (Re | Im,
//                      128 columns each), releasing stages through tcgen05.commit on empty[stage]
//                      and finished chunks on accfull[buffer];
//   warps 0-3:         drain each finished chunk (TMEM lanes = tile rows) into int64 accumulators
//                      kept in TMEM (low words in columns 256..383, high words in 384..511) and
//                      release the buffer on accempty[buffer], so the next chunk's products run
//                      meanwhile; at the end they scale the sums and write G.
// Every wait is bounded and also ends on a shared abort flag; a time-out sets *err and the CTA
// frees its TMEM and leaves.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>

#include "mmf_internal.h"
#include "umma_common.h"

#define OZ_W 8                 // bits per slice
#define OZ_L 4                 // pairs a + b <= OZ_L
#define OZ_SCALE 256.f         // 2^OZ_W
#define OZ_NMAX 60000          // int64 range of the Gram sums (2n <= 2^17)
#define OZ_THREADS 128
#define OZ_TM 128
#define OZ_TN 64
#define OZ_KSTEP 64            // BF16 elements of K per stage (one 128-byte row segment)
#define OZ_KCH (16 * OZ_KSTEP) // K per exact FP32 accumulation: 1024 * 2^14 = 2^24
#define OZ_STAGE_BYTES (16384 + 8192 + 8192)
#define OZ_STAGES 6
#define OZ_TILE_ELEMS 4096      // one 64 x 64 BF16 tile (8 KB)
#define OZ_WARPS 6

static_assert(OZ_S == OZ_L + 1, "slices cover the kept pairs");

__host__ __device__ __forceinline__ int oz_la(int n) { return (2 * n + OZ_KSTEP - 1) / OZ_KSTEP * OZ_KSTEP; }
__host__ __device__ __forceinline__ int oz_nt(int n) { return oz_la(n) / OZ_KSTEP; }             // K tiles
__host__ __device__ __forceinline__ int oz_nq(int n) { return ((n + 63) / 64 + 1) / 2 * 2; }     // 64-row panels
// element offset of tile (slice s, K tile t, row panel q); A tiles (128 rows) are panels 2I, 2I+1
__host__ __device__ __forceinline__ int64_t oz_tile_off(int n, int s, int t, int q) {
    return (((int64_t)s * oz_nt(n) + t) * oz_nq(n) + q) * OZ_TILE_ELEMS;
}

// ------------------------------------------------------------------ slicing
// One warp per row i of the slice matrices (column i of X1; rows past n are zero): the scale
// exponent, then for each 16-byte chunk of 8 K entries the OZ_S slices of a_i and a'_i, written
// at their swizzled place in the tile.
__global__ void __launch_bounds__(256) k_oz_slice(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                  const float2* __restrict__ X1g, __nv_bfloat16* __restrict__ S,
                                                  int* __restrict__ expg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = oz_la(n);
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= oz_nq(n) * 64) return;
    const bool live = i < n;
    const float2* x = X1g + d.mat_off + (int64_t)(live ? i : 0) * d.ld;
    float m = 0.f;
    if (live)
        for (int k = lane; k < n; k += 32) m = fmaxf(m, fmaxf(fabsf(x[k].x), fabsf(x[k].y)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    int e = 0;
    if (m > 0.f) frexpf(m, &e);  // m = f 2^e, f in [0.5, 1): |x| 2^-(e+1) < 1/2
    if (live && lane == 0) expg[d.vec_off + i] = e;
    __nv_bfloat16* Sys = S + d.oz_off;
    const int q = i >> 6, r = i & 63;
    for (int jc = lane; jc < la / 8; jc += 32) {
        const int k0 = jc * 8;
        float ta[8], tb[8];  // scaled entries of a_i and a'_i
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            float va = 0.f, vb = 0.f;
            if (live && k < 2 * n) {
                if (k < n) {
                    va = x[k].x;   // Re x_ki
                    vb = x[k].y;   // Im x_ki
                } else {
                    va = x[k - n].y;   // Im x_ki
                    vb = -x[k - n].x;  // -Re x_ki
                }
            }
            ta[u] = ldexpf(va, -(e + 1));
            tb[u] = ldexpf(vb, -(e + 1));
        }
        const int t = k0 >> 6, j = (k0 & 63) >> 3;
        const int64_t inner = (int64_t)(r >> 3) * 512 + (r & 7) * 64 + ((j ^ (r & 7)) << 3);  // BF16 units
#pragma unroll
        for (int sl = 0; sl < OZ_S; ++sl) {
            uint32_t pa[4], pb[4];
#pragma unroll
            for (int u = 0; u < 8; u += 2) {
                float a0 = ta[u] * OZ_SCALE, a1 = ta[u + 1] * OZ_SCALE, b0 = tb[u] * OZ_SCALE, b1 = tb[u + 1] * OZ_SCALE;
                const float ra0 = rintf(a0), ra1 = rintf(a1), rb0 = rintf(b0), rb1 = rintf(b1);
                ta[u] = a0 - ra0;
                ta[u + 1] = a1 - ra1;
                tb[u] = b0 - rb0;
                tb[u + 1] = b1 - rb1;
                const __nv_bfloat162 ha = __floats2bfloat162_rn(ra0, ra1), hb = __floats2bfloat162_rn(rb0, rb1);
                pa[u >> 1] = *reinterpret_cast<const uint32_t*>(&ha);
                pb[u >> 1] = *reinterpret_cast<const uint32_t*>(&hb);
            }
            *reinterpret_cast<uint4*>(Sys + oz_tile_off(n, sl, t, q) + inner) = make_uint4(pa[0], pa[1], pa[2], pa[3]);
            *reinterpret_cast<uint4*>(Sys + oz_tile_off(n, OZ_S + sl, t, q) + inner) =
                make_uint4(pb[0], pb[1], pb[2], pb[3]);
        }
    }
}

// ------------------------------------------------------------------ products
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

#define OZ_TMEM_COLS 512u
#define OZ_COL_LO 256   // int64 accumulators in TMEM: low words (Re 256..319, Im 320..383)
#define OZ_COL_HI 384   //                               high words (Re 384..447, Im 448..511)

__device__ __forceinline__ void tm_ld32(uint32_t ta, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
        "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
}
__device__ __forceinline__ void tm_st32(uint32_t ta, const uint32_t* v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]),
        "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]),
        "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
        : "memory");
}

// bounded wait that also gives up when another role has aborted; sets the abort flag on time-out
__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const uint32_t a = smem_u32(bar);
    for (uint32_t it = 0; it < UM_WAIT_LIMIT; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((it & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    return false;
}

__device__ __forceinline__ void oz_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(OZ_WARPS * 32, 1) k_oz_gram(const MmfDesc* __restrict__ descs,
                                                              const int* __restrict__ idx,
                                                              const __nv_bfloat16* __restrict__ S,
                                                              const int* __restrict__ expg, double2* __restrict__ Gg,
                                                              int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ uint64_t full[OZ_STAGES], empty[OZ_STAGES], accfull[2], accempty[2];
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = oz_la(n);
    int I, J;
    if (!oz_tile(blockIdx.x, n, I, J)) return;
    const int i0 = I * OZ_TM, j0 = J * OZ_TN;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    volatile int* abort_flag = &abort_s;
    if (threadIdx.x == 0) {
        abort_s = 0;
        for (int q = 0; q < OZ_STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accfull[q], 1);
            mbar_init(&accempty[q], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int nkc = (la + OZ_KCH - 1) / OZ_KCH;      // K chunks per pair
    const int npairs = (OZ_L + 1) * (OZ_L + 2) / 2;  // pairs a + b <= OZ_L
    const int nchunks = npairs * nkc;
    const __nv_bfloat16* Sys = S + d.oz_off;
    const int nt = oz_nt(n);

    if (warp == 4) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int a = 0; a <= OZ_L; ++a)
                for (int b = 0; a + b <= OZ_L; ++b)
                    for (int t = 0; t < nt; ++t, ++it) {
                        const int st = (int)(it % OZ_STAGES);
                        const uint32_t use = it / OZ_STAGES;
                        if (use > 0 && !oz_wait(&empty[st], (use - 1) & 1u, abort_flag)) goto producer_done;
                        const uint32_t fb = smem_u32(&full[st]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"((uint32_t)OZ_STAGE_BYTES)
                                     : "memory");
                        const uint32_t dst = sbase + (uint32_t)st * OZ_STAGE_BYTES;
                        const __nv_bfloat16* srcA = Sys + oz_tile_off(n, a, t, 2 * I);
                        const __nv_bfloat16* srcB = Sys + oz_tile_off(n, b, t, J);
                        const __nv_bfloat16* srcBp = Sys + oz_tile_off(n, OZ_S + b, t, J);
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst),
                            "l"(srcA), "r"(16384u), "r"(fb)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + 16384u),
                            "l"(srcB), "r"(8192u), "r"(fb)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + 24576u),
                            "l"(srcBp), "r"(8192u), "r"(fb)
                            : "memory");
                    }
        producer_done:;
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_mn(1, OZ_TM, OZ_TN);
            uint32_t it = 0;
            int c = 0;
            bool ok = true;
            for (int p = 0; p < npairs && ok; ++p)
                for (int kc = 0; kc < nkc && ok; ++kc, ++c) {
                    const int buf = c & 1;
                    const uint32_t v = (uint32_t)c >> 1;
                    if (v > 0 && !oz_wait(&accempty[buf], (v - 1) & 1u, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dre = tmem + (uint32_t)buf * 128u, dim = dre + OZ_TN;
                    const int t0 = kc * (OZ_KCH / OZ_KSTEP), t1 = min(nt, t0 + OZ_KCH / OZ_KSTEP);
                    for (int t = t0; t < t1; ++t, ++it) {
                        const int st = (int)(it % OZ_STAGES);
                        if (!oz_wait(&full[st], (it / OZ_STAGES) & 1u, abort_flag)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = sbase + (uint32_t)st * OZ_STAGE_BYTES;
                        const uint64_t da = umma_desc(sa), db = umma_desc(sa + 16384u), dbp = umma_desc(sa + 24576u);
#pragma unroll
                        for (int q = 0; q < OZ_KSTEP / 16; ++q) {  // 32 bytes of K per instruction
                            const uint32_t accf = (t > t0 || q > 0) ? 1u : 0u;
                            const uint64_t adv = (uint64_t)((q * 32) >> 4);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dre),
                                "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(accf)
                                : "memory");
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dim),
                                "l"(da + adv), "l"(dbp + adv), "r"(idesc), "r"(accf)
                                : "memory");
                        }
                        oz_commit(&empty[st]);  // the stage is free once these MMAs have read it
                    }
                    if (!ok) break;
                    oz_commit(&accfull[buf]);  // the chunk's sums are complete
                }
        }
    } else {
        // ---------------------------------------------------------------- drain (warps 0-3)
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        {
            uint32_t z[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) z[q] = 0u;
#pragma unroll 1
            for (int col = OZ_COL_LO; col < OZ_COL_HI + 2 * OZ_TN; col += 32) tm_st32(trow + (uint32_t)col, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        int c = 0;
        bool ok = true;
        for (int a = 0; a <= OZ_L && ok; ++a)
            for (int b = 0; a + b <= OZ_L && ok; ++b) {
                const int sh = OZ_W * (OZ_L - a - b);
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int buf = c & 1;
                    if (!oz_wait(&accfull[buf], ((uint32_t)c >> 1) & 1u, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                    for (int g = 0; g < 2 * OZ_TN; g += 32) {
                        uint32_t v[32], lo[32], hi[32];
                        tm_ld32(trow + (uint32_t)(buf * 128 + g), v);
                        tm_ld32(trow + (uint32_t)(OZ_COL_LO + g), lo);
                        tm_ld32(trow + (uint32_t)(OZ_COL_HI + g), hi);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const long long iv = __float2ll_rn(__uint_as_float(v[q]));  // an exact integer
                            const long long term = sh >= 0 ? (iv << sh) : (iv >> (-sh));
                            const long long acc64 = (long long)(((unsigned long long)hi[q] << 32) | lo[q]) + term;
                            lo[q] = (uint32_t)(unsigned long long)acc64;
                            hi[q] = (uint32_t)((unsigned long long)acc64 >> 32);
                        }
                        tm_st32(trow + (uint32_t)(OZ_COL_LO + g), lo);
                        tm_st32(trow + (uint32_t)(OZ_COL_HI + g), hi);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[buf]))
                                 : "memory");
                }
            }
        (void)nchunks;
        if (ok) {
            const int i = i0 + warp * 32 + lane;
            const int ei = i < n ? expg[d.vec_off + i] : 0;
            double2* G = Gg + d.mat_off;
#pragma unroll 1
            for (int g = 0; g < OZ_TN; g += 32) {
                uint32_t rlo[32], rhi[32], ilo[32], ihi[32];
                tm_ld32(trow + (uint32_t)(OZ_COL_LO + g), rlo);
                tm_ld32(trow + (uint32_t)(OZ_COL_HI + g), rhi);
                tm_ld32(trow + (uint32_t)(OZ_COL_LO + OZ_TN + g), ilo);
                tm_ld32(trow + (uint32_t)(OZ_COL_HI + OZ_TN + g), ihi);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int j = j0 + g + q;
                    if (i < n && j <= i) {  // j <= i < n
                        const int sc = ei + expg[d.vec_off + j] + 2 - OZ_W * (OZ_L + 2);
                        const long long ar = (long long)(((unsigned long long)rhi[q] << 32) | rlo[q]);
                        const long long ai = (long long)(((unsigned long long)ihi[q] << 32) | ilo[q]);
                        const double gr = ldexp((double)ar, sc);
                        const double gi = (i == j) ? 0.0 : ldexp((double)ai, sc);
                        G[(int64_t)j * d.ld + i] = make_double2(gr, gi);
                        if (i != j) G[(int64_t)i * d.ld + j] = make_double2(gr, -gi);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && abort_s) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
}

size_t mmf_ozaki_slice_elems(int n) { return (size_t)2 * OZ_S * oz_nt(n) * oz_nq(n) * OZ_TILE_ELEMS; }

int mmf_ozaki_max_n() { return OZ_NMAX; }

cudaError_t mmf_launch_ozaki_gram(const MmfLaunch& L, const float2* X1, void* S, int* exps, double2* G, int* err) {
    if (L.count <= 0) return cudaSuccess;
    if (L.nmax > OZ_NMAX) return cudaErrorInvalidValue;
    const int rows = oz_nq(L.nmax) * 64;
    k_oz_slice<<<dim3((rows + 7) / 8, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X1, (__nv_bfloat16*)S, exps);
    const int nI = (L.nmax + OZ_TM - 1) / OZ_TM, nJ = (L.nmax + OZ_TN - 1) / OZ_TN;
    int tiles = 0;
    for (int I = 0; I < nI; ++I) tiles += std::min(2 * I + 2, nJ);
    const size_t sm = (size_t)OZ_STAGES * OZ_STAGE_BYTES + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_oz_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_oz_gram<<<dim3(tiles, L.count), OZ_WARPS * 32, sm, L.stream>>>(L.desc, L.idx, (const __nv_bfloat16*)S, exps, G,
                                                                      err);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ time evolution (Eq. 3-5)
// Phi_j(t, l) = sum_b F(t, b) Z[(j, b), l] for every level j, eigenvector l and time t, by the
// same exact slicing: A rows r = j n + l hold a_r = [Re Z((j, b), l) | Im Z((j, b), l)] over b
// (K = 2M), B rows t hold [Re F(t, b) | -Im F(t, b)] and B' rows [Im F(t, b) | Re F(t, b)], so
// that a_r . b_t = Re Phi and a_r . b'_t = Im Phi.  Z (FP64) is sliced from its FP32 pieces
// Z1 + Zlo in double-FP32 (each step 256 t - rint(256 t) exact, the pair renormalised by TwoSum),
// F from its pre-split phase table.  Phi goes to FP64 (error below ~2^-38 of each row's largest
// |Z| times sum_b |F|); U(t, t0)[j, i] = sum_l Phi_j(t, l) e^{-i E_l (t - t0)} conj(Z[(i, b0), l])
// follows in FP64.  The operands and Phi live in the system's operand area.
struct PhiLayout {
    int ra, nqa, nqb, ntk;           // A rows (D n), 64-row panels of A (even) and B, K tiles
    int64_t sa, sb, ea, eb, phi, total;  // offsets in BF16 units from the area's start
};
__host__ __device__ inline PhiLayout phi_layout(int n, int D, int M, int nt) {
    PhiLayout o;
    o.ra = D * n;
    o.nqa = ((o.ra + 63) / 64 + 1) / 2 * 2;
    o.nqb = (nt + 63) / 64;
    o.ntk = (2 * M + OZ_KSTEP - 1) / OZ_KSTEP;
    o.sa = 0;
    o.sb = o.sa + (int64_t)OZ_S * o.ntk * o.nqa * OZ_TILE_ELEMS;
    o.ea = o.sb + (int64_t)2 * OZ_S * o.ntk * o.nqb * OZ_TILE_ELEMS;  // int exponents of A rows
    o.eb = o.ea + (int64_t)2 * o.nqa * 64;                             // int exponents of B rows
    o.phi = (o.eb + (int64_t)2 * o.nqb * 64 + 7) / 8 * 8;              // double2, 16-byte aligned
    o.total = o.phi + (int64_t)8 * o.ra * nt;
    return o;
}

// place of the 16-byte chunk j (K entries 8j .. 8j+7 of a 64-K tile) of row r in a 64-row panel
__device__ __forceinline__ int64_t oz_inner(int r, int j) {
    return (int64_t)(r >> 3) * 512 + (r & 7) * 64 + ((j ^ (r & 7)) << 3);
}

// OZ_S slices of eight scaled entries given as double-FP32 pairs (t1 + t2, |t1 + t2| < 1)
__device__ __forceinline__ void oz_slices8(float* t1, float* t2, uint4* out) {
#pragma unroll
    for (int sl = 0; sl < OZ_S; ++sl) {
        uint32_t pk[4];
#pragma unroll
        for (int u = 0; u < 8; u += 2) {
            float v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float x = t1[u + h] * OZ_SCALE;  // exact
                const float r = rintf(x);
                const float a = x - r;               // exact
                const float b = t2[u + h] * OZ_SCALE;  // exact
                const float s = a + b;               // TwoSum: (s, err) = a + b exactly
                const float bb = s - a;
                t1[u + h] = s;
                t2[u + h] = (a - (s - bb)) + (b - bb);
                v[h] = r;
            }
            const __nv_bfloat162 hv = __floats2bfloat162_rn(v[0], v[1]);
            pk[u >> 1] = *reinterpret_cast<const uint32_t*>(&hv);
        }
        out[sl] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
    }
}

// A slices: one warp per row r = j n + l (rows past D n are zero)
__global__ void __launch_bounds__(256) k_phi_slice_a(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                     const float2* __restrict__ Z1g, const float2* __restrict__ Zlog,
                                                     uint16_t* __restrict__ pool, int nt) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const PhiLayout o = phi_layout(d.n, d.D, d.M, nt);
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= o.nqa * 64) return;
    uint16_t* W = pool + d.oz_off;
    const bool live = r < o.ra;
    const int j = live ? r / d.n : 0, l = live ? r - j * d.n : 0;
    const float2* z1 = Z1g + d.mat_off + (int64_t)l * d.ld + j;
    const float2* zl = Zlog + d.mat_off + (int64_t)l * d.ld + j;
    const int M = d.M, D = d.D;
    float m = 0.f;
    if (live)
        for (int b = lane; b < M; b += 32) {
            const float2 z = z1[b * D];
            m = fmaxf(m, fmaxf(fabsf(z.x), fabsf(z.y)));
        }
    for (int q = 16; q > 0; q >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, q));
    int e = 0;
    if (m > 0.f) frexpf(m, &e);  // |z| 2^-(e+1) < 1/2 (also for z1 + zlo, see the comment above)
    if (live && lane == 0) reinterpret_cast<int*>(W + o.ea)[r] = e;
    const float sc = ldexpf(1.f, -(e + 1));
    __nv_bfloat16* SA = reinterpret_cast<__nv_bfloat16*>(W + o.sa);
    const int q = r >> 6, rr = r & 63;
    for (int jc = lane; jc < o.ntk * 8; jc += 32) {
        const int k0 = jc * 8;
        float t1[8], t2[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            float a = 0.f, b = 0.f;
            if (live && k < 2 * M) {
                const int bb = k < M ? k : k - M;
                const float2 h = z1[bb * D], lo = zl[bb * D];
                a = k < M ? h.x : h.y;
                b = k < M ? lo.x : lo.y;
            }
            t1[u] = a * sc;
            t2[u] = b * sc;
        }
        uint4 sl[OZ_S];
        oz_slices8(t1, t2, sl);
        const int t = k0 >> 6, jj = (k0 & 63) >> 3;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s)
            *reinterpret_cast<uint4*>(SA + (((int64_t)s * o.ntk + t) * o.nqa + q) * OZ_TILE_ELEMS + oz_inner(rr, jj)) =
                sl[s];
    }
}

// B and B' slices from the phase table (F[t][b] in FP32 pieces): one warp per time row
__global__ void __launch_bounds__(256) k_phi_slice_b(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                     const Split* __restrict__ Fg, uint16_t* __restrict__ pool,
                                                     int nt) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const PhiLayout o = phi_layout(d.n, d.D, d.M, nt);
    const int lane = threadIdx.x & 31;
    const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (t >= o.nqb * 64) return;
    uint16_t* W = pool + d.oz_off;
    const bool live = t < nt;
    const Split* F = Fg + d.f_off + (int64_t)(live ? t : 0) * d.M;
    const int M = d.M;
    float m = 0.f;
    if (live)
        for (int b = lane; b < M; b += 32) m = fmaxf(m, fmaxf(fabsf(F[b].r1), fabsf(F[b].i1)));
    for (int q = 16; q > 0; q >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, q));
    int e = 0;
    if (m > 0.f) frexpf(m, &e);
    if (live && lane == 0) reinterpret_cast<int*>(W + o.eb)[t] = e;
    const float sc = ldexpf(1.f, -(e + 1));
    __nv_bfloat16* SB = reinterpret_cast<__nv_bfloat16*>(W + o.sb);
    const int q = t >> 6, rr = t & 63;
    for (int jc = lane; jc < o.ntk * 8; jc += 32) {
        const int k0 = jc * 8;
        float a1[8], a2[8], c1[8], c2[8];  // B (Re F | -Im F) and B' (Im F | Re F)
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int k = k0 + u;
            float x1 = 0.f, x2 = 0.f, y1 = 0.f, y2 = 0.f;
            if (live && k < 2 * M) {
                const Split f = F[k < M ? k : k - M];
                if (k < M) { x1 = f.r1; x2 = f.r2; y1 = f.i1; y2 = f.i2; }
                else       { x1 = -f.i1; x2 = -f.i2; y1 = f.r1; y2 = f.r2; }
            }
            a1[u] = x1 * sc; a2[u] = x2 * sc;
            c1[u] = y1 * sc; c2[u] = y2 * sc;
        }
        uint4 sl[OZ_S];
        const int tk = k0 >> 6, jj = (k0 & 63) >> 3;
        oz_slices8(a1, a2, sl);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s)
            *reinterpret_cast<uint4*>(SB + (((int64_t)s * o.ntk + tk) * o.nqb + q) * OZ_TILE_ELEMS + oz_inner(rr, jj)) =
                sl[s];
        oz_slices8(c1, c2, sl);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s)
            *reinterpret_cast<uint4*>(SB + (((int64_t)(OZ_S + s) * o.ntk + tk) * o.nqb + q) * OZ_TILE_ELEMS +
                                      oz_inner(rr, jj)) = sl[s];
    }
}

// Phi on the tensor cores: one CTA per 128 (rows r) x 64 (times) tile, roles as in k_oz_gram
__global__ void __launch_bounds__(OZ_WARPS * 32, 1) k_oz_phi(const MmfDesc* __restrict__ descs,
                                                             const int* __restrict__ idx, uint16_t* __restrict__ pool,
                                                             int nt, int nqb_max, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char oz_smem[];
    __shared__ uint64_t full[OZ_STAGES], empty[OZ_STAGES], accfull[2], accempty[2];
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    const MmfDesc d = descs[idx[blockIdx.y]];
    const PhiLayout o = phi_layout(d.n, d.D, d.M, nt);
    const int I = blockIdx.x / nqb_max, J = blockIdx.x - I * nqb_max;
    if (2 * I >= o.nqa || J >= o.nqb) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)oz_smem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    volatile int* abort_flag = &abort_s;
    if (threadIdx.x == 0) {
        abort_s = 0;
        for (int q = 0; q < OZ_STAGES; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accfull[q], 1);
            mbar_init(&accempty[q], 128);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(OZ_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int la = o.ntk * OZ_KSTEP;
    const int nkc = (la + OZ_KCH - 1) / OZ_KCH;      // K chunks per pair
    const int npairs = (OZ_L + 1) * (OZ_L + 2) / 2;  // pairs a + b <= OZ_L
    const uint16_t* W = pool + d.oz_off;
    const __nv_bfloat16* SA = reinterpret_cast<const __nv_bfloat16*>(W + o.sa);
    const __nv_bfloat16* SB = reinterpret_cast<const __nv_bfloat16*>(W + o.sb);
    const int ntk = o.ntk;

    if (warp == 4) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            uint32_t it = 0;
            for (int a = 0; a <= OZ_L; ++a)
                for (int b = 0; a + b <= OZ_L; ++b)
                    for (int t = 0; t < ntk; ++t, ++it) {
                        const int st = (int)(it % OZ_STAGES);
                        const uint32_t use = it / OZ_STAGES;
                        if (use > 0 && !oz_wait(&empty[st], (use - 1) & 1u, abort_flag)) goto phi_producer_done;
                        const uint32_t fb = smem_u32(&full[st]);
                        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                                     "r"((uint32_t)OZ_STAGE_BYTES)
                                     : "memory");
                        const uint32_t dst = sbase + (uint32_t)st * OZ_STAGE_BYTES;
                        const __nv_bfloat16* srcA = SA + (((int64_t)a * ntk + t) * o.nqa + 2 * I) * OZ_TILE_ELEMS;
                        const __nv_bfloat16* srcB = SB + (((int64_t)b * ntk + t) * o.nqb + J) * OZ_TILE_ELEMS;
                        const __nv_bfloat16* srcBp =
                            SB + (((int64_t)(OZ_S + b) * ntk + t) * o.nqb + J) * OZ_TILE_ELEMS;
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst),
                            "l"(srcA), "r"(16384u), "r"(fb)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + 16384u),
                            "l"(srcB), "r"(8192u), "r"(fb)
                            : "memory");
                        asm volatile(
                            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                dst + 24576u),
                            "l"(srcBp), "r"(8192u), "r"(fb)
                            : "memory");
                    }
        phi_producer_done:;
        }
    } else if (warp == 5) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_mn(1, OZ_TM, OZ_TN);
            uint32_t it = 0;
            int c = 0;
            bool ok = true;
            for (int p = 0; p < npairs && ok; ++p)
                for (int kc = 0; kc < nkc && ok; ++kc, ++c) {
                    const int buf = c & 1;
                    const uint32_t v = (uint32_t)c >> 1;
                    if (v > 0 && !oz_wait(&accempty[buf], (v - 1) & 1u, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t dre = tmem + (uint32_t)buf * 128u, dim = dre + OZ_TN;
                    const int t0 = kc * (OZ_KCH / OZ_KSTEP), t1 = min(ntk, t0 + OZ_KCH / OZ_KSTEP);
                    for (int t = t0; t < t1; ++t, ++it) {
                        const int st = (int)(it % OZ_STAGES);
                        if (!oz_wait(&full[st], (it / OZ_STAGES) & 1u, abort_flag)) { ok = false; break; }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = sbase + (uint32_t)st * OZ_STAGE_BYTES;
                        const uint64_t da = umma_desc(sa), db = umma_desc(sa + 16384u), dbp = umma_desc(sa + 24576u);
#pragma unroll
                        for (int q = 0; q < OZ_KSTEP / 16; ++q) {  // 32 bytes of K per instruction
                            const uint32_t accf = (t > t0 || q > 0) ? 1u : 0u;
                            const uint64_t adv = (uint64_t)((q * 32) >> 4);
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dre),
                                "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(accf)
                                : "memory");
                            asm volatile(
                                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dim),
                                "l"(da + adv), "l"(dbp + adv), "r"(idesc), "r"(accf)
                                : "memory");
                        }
                        oz_commit(&empty[st]);
                    }
                    if (!ok) break;
                    oz_commit(&accfull[buf]);
                }
        }
    } else {
        // ---------------------------------------------------------------- drain (warps 0-3)
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
        {
            uint32_t z[32];
#pragma unroll
            for (int q = 0; q < 32; ++q) z[q] = 0u;
#pragma unroll 1
            for (int col = OZ_COL_LO; col < OZ_COL_HI + 2 * OZ_TN; col += 32) tm_st32(trow + (uint32_t)col, z);
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        int c = 0;
        bool ok = true;
        for (int a = 0; a <= OZ_L && ok; ++a)
            for (int b = 0; a + b <= OZ_L && ok; ++b) {
                const int sh = OZ_W * (OZ_L - a - b);
                for (int kc = 0; kc < nkc; ++kc, ++c) {
                    const int buf = c & 1;
                    if (!oz_wait(&accfull[buf], ((uint32_t)c >> 1) & 1u, abort_flag)) { ok = false; break; }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
                    for (int g = 0; g < 2 * OZ_TN; g += 32) {
                        uint32_t v[32], lo[32], hi[32];
                        tm_ld32(trow + (uint32_t)(buf * 128 + g), v);
                        tm_ld32(trow + (uint32_t)(OZ_COL_LO + g), lo);
                        tm_ld32(trow + (uint32_t)(OZ_COL_HI + g), hi);
                        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                        for (int q = 0; q < 32; ++q) {
                            const long long iv = __float2ll_rn(__uint_as_float(v[q]));  // an exact integer
                            const long long term = sh >= 0 ? (iv << sh) : (iv >> (-sh));
                            const long long acc64 = (long long)(((unsigned long long)hi[q] << 32) | lo[q]) + term;
                            lo[q] = (uint32_t)(unsigned long long)acc64;
                            hi[q] = (uint32_t)((unsigned long long)acc64 >> 32);
                        }
                        tm_st32(trow + (uint32_t)(OZ_COL_LO + g), lo);
                        tm_st32(trow + (uint32_t)(OZ_COL_HI + g), hi);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[buf]))
                                 : "memory");
                }
            }
        if (ok) {
            const int r = I * OZ_TM + warp * 32 + lane;
            const int* ea = reinterpret_cast<const int*>(W + o.ea);
            const int* eb = reinterpret_cast<const int*>(W + o.eb);
            double2* Phi = reinterpret_cast<double2*>(pool + d.oz_off + o.phi);
            const int er = r < o.ra ? ea[r] : 0;
#pragma unroll 1
            for (int g = 0; g < OZ_TN; g += 32) {
                uint32_t rlo[32], rhi[32], ilo[32], ihi[32];
                tm_ld32(trow + (uint32_t)(OZ_COL_LO + g), rlo);
                tm_ld32(trow + (uint32_t)(OZ_COL_HI + g), rhi);
                tm_ld32(trow + (uint32_t)(OZ_COL_LO + OZ_TN + g), ilo);
                tm_ld32(trow + (uint32_t)(OZ_COL_HI + OZ_TN + g), ihi);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (r < o.ra) {
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        const int t = J * OZ_TN + g + q;
                        if (t < nt) {
                            const int sc = er + eb[t] + 2 - OZ_W * (OZ_L + 2);
                            const long long ar = (long long)(((unsigned long long)rhi[q] << 32) | rlo[q]);
                            const long long ai = (long long)(((unsigned long long)ihi[q] << 32) | ilo[q]);
                            Phi[(int64_t)r * nt + t] = make_double2(ldexp((double)ar, sc), ldexp((double)ai, sc));
                        }
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && abort_s) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(OZ_TMEM_COLS)
                     : "memory");
}

// U(t, t0)[j, i] += sum over the CTA's 32 eigenvectors l of Phi_j(t, l) e^{-i E_l (t - t0)} conj(Z0(i, l)),
// FP64; CTA (eigenvector chunk, 64-time chunk); thread (t, j) keeps the D sums over i
#define PU_L 32
#define PU_T 64
#define PU_DMAX 16  // levels per system on this path (more take the double-FP32 kernel)
__global__ void __launch_bounds__(256) k_phi_u(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                               const uint16_t* __restrict__ pool, const double* __restrict__ Eg,
                                               const double2* __restrict__ Zg, const double* __restrict__ tpool,
                                               double t0, int nt, double2* __restrict__ U) {
    __shared__ double2 ph[PU_L][PU_T];
    __shared__ double2 z0[PU_L][PU_DMAX];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, D = d.D;
    const int l0 = blockIdx.x * PU_L, tb = blockIdx.y * PU_T;
    if (l0 >= n || tb >= nt) return;
    const int nl = min(PU_L, n - l0), ntt = min(PU_T, nt - tb);
    const PhiLayout o = phi_layout(n, D, d.M, nt);
    const double2* Phi = reinterpret_cast<const double2*>(pool + d.oz_off + o.phi);
    for (int e = threadIdx.x; e < PU_L * PU_T; e += blockDim.x) {
        const int a = e / PU_T, tt = e - a * PU_T;
        double s = 0.0, c = 1.0;
        if (a < nl && tt < ntt) sincos(Eg[d.vec_off + l0 + a] * (tpool[d.t_off + tb + tt] - t0), &s, &c);
        ph[a][tt] = make_double2(c, -s);
    }
    for (int e = threadIdx.x; e < PU_L * D; e += blockDim.x) {
        const int a = e / D, i = e - a * D;
        z0[a][i] = a < nl ? Zg[d.mat_off + (int64_t)(l0 + a) * d.ld + i + D * d.b0] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int task = threadIdx.x; task < ntt * D; task += blockDim.x) {
        const int tt = task % ntt, j = task / ntt;
        double2 acc[PU_DMAX];
#pragma unroll
        for (int i = 0; i < PU_DMAX; ++i) acc[i] = make_double2(0.0, 0.0);
        for (int a = 0; a < nl; ++a) {
            const double2 f = Phi[((int64_t)j * n + l0 + a) * nt + tb + tt] * ph[a][tt];
#pragma unroll
            for (int i = 0; i < PU_DMAX; ++i)
                if (i < D) acc[i] = acc[i] + cmulc(z0[a][i], f);
        }
        double2* u = U + d.u_off + ((int64_t)(tb + tt) * D + j) * D;
#pragma unroll
        for (int i = 0; i < PU_DMAX; ++i)
            if (i < D) {
                atomicAdd(&u[i].x, acc[i].x);
                atomicAdd(&u[i].y, acc[i].y);
            }
    }
}

int64_t mmf_phi_elems(int n, int D, int M, int nt) { return phi_layout(n, D, M, nt).total; }

int mmf_phi_max_levels() { return PU_DMAX; }

cudaError_t mmf_launch_phi(const MmfLaunch& L, int Dmax, int nt, const float2* Z1, const float2* Zlo,
                           const void* F, const double* E, const double2* Z, const double* t, double t0, void* pool,
                           double2* U, int* err) {
    if (L.count <= 0 || nt <= 0) return cudaSuccess;
    if (Dmax > PU_DMAX) return cudaErrorInvalidValue;
    uint16_t* P = (uint16_t*)pool;
    const int rowsA = ((Dmax * L.nmax + 63) / 64 + 1) / 2 * 2 * 64;
    const int nqb = (nt + 63) / 64;
    k_phi_slice_a<<<dim3((rowsA + 7) / 8, L.count), 256, 0, L.stream>>>(L.desc, L.idx, Z1, Zlo, P, nt);
    k_phi_slice_b<<<dim3(nqb * 8, L.count), 256, 0, L.stream>>>(L.desc, L.idx, (const Split*)F, P, nt);
    const size_t sm = (size_t)OZ_STAGES * OZ_STAGE_BYTES + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_oz_phi, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nI = rowsA / 128;
    k_oz_phi<<<dim3(nI * nqb, L.count), OZ_WARPS * 32, sm, L.stream>>>(L.desc, L.idx, P, nt, nqb, err);
    k_phi_u<<<dim3((L.nmax + PU_L - 1) / PU_L, (nt + PU_T - 1) / PU_T, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, P, E, Z, t, t0, nt, U);
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
