// k_umma.cu -- batched GEMM on the 5th-generation tensor cores (tcgen05 / TMEM).
//
//   C[b](m, n) = sum_{p < P} sum_k A_p[b](m, k) * B_p[b](n, k)        (FP32 accumulation)
//
// Operands are K-major (k contiguous) in global memory, element type TF32 (FP32 storage, low 13
// mantissa bits zero) or BF16.  One CTA of 128 threads computes a 128 x 128 tile of C for one
// batch entry: operand tiles of 128 rows x 128 bytes are staged by cp.async into shared memory
// in the 128-byte-swizzled K-major layout (8-row atoms of 1 KB, 16-byte chunk j of row r at
// position j ^ (r mod 8)), one elected thread issues tcgen05.mma (M = 128, N = 128) into a TMEM
// accumulator and commits to an mbarrier, two stages are in flight, and the four warps read
// the accumulator back with tcgen05.ld (warp w owns TMEM lanes 32w..32w+31 = rows of C).
// Several products (P <= 3) share the accumulator, which is how a split-precision product such
// as A1 B1 + A1 B2 + A2 B1 (TF32 pieces of FP32 data) is formed in one pass.
// Every mbarrier wait is bounded; on time-out the CTA sets *err and leaves after freeing TMEM.
#include <cuda_bf16.h>

#include <cstring>

#include "mmf_internal.h"
#include "umma_common.h"

#define UM_THREADS 128
#define UM_TILE 128           // M and N of one tile
#define UM_KB 128             // bytes of K per stage and row (one swizzle atom width)
#define UM_STAGES 2


template <int ESZ>
__device__ __forceinline__ void load_tile(uint32_t sbase, const unsigned char* g, int rows_valid,
                                          int k0_bytes, int kbytes_valid, int64_t ld_bytes) {
    // 128 rows x 128 bytes = 1024 chunks of 16 bytes, 8 per thread
    for (int c = threadIdx.x; c < UM_TILE * (UM_KB / 16); c += UM_THREADS) {
        const int r = c >> 3, j = c & 7;
        const uint32_t dst = sbase + (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
        const int kb = k0_bytes + j * 16;
        int bytes = 0;
        const unsigned char* src = g;
        if (r < rows_valid && kb < kbytes_valid) {
            bytes = min(16, kbytes_valid - kb);
            src = g + (int64_t)r * ld_bytes + kb;
        }
        cp_async16(dst, src, bytes);
    }
}

template <int KIND>  // 0: kind::tf32 (4-byte elements), 1: kind::f16 with BF16 (2-byte elements)
__global__ void __launch_bounds__(UM_THREADS, 1) k_umma_gemm(const UmmaJob* __restrict__ jobs, int P,
                                                             int* __restrict__ err) {
    constexpr int ESZ = KIND == 0 ? 4 : 2;
    extern __shared__ __align__(1024) unsigned char um_smem[];
    __shared__ uint64_t bar[UM_STAGES];
    __shared__ uint32_t tmem_base_s;
    const UmmaJob jb = jobs[blockIdx.z];
    const int m0 = blockIdx.x * UM_TILE, n0 = blockIdx.y * UM_TILE;
    if (m0 >= jb.M || n0 >= jb.N) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // shared layout per stage: P A-tiles then P B-tiles, 16 KB each, 1 KB aligned
    unsigned char* base = (unsigned char*)(((uintptr_t)um_smem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    const uint32_t stage_bytes = 2u * P * 16384u;

    if (threadIdx.x == 0) {
        for (int s = 0; s < UM_STAGES; ++s) mbar_init(&bar[s], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_s)),
                     "r"(128u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base_s;

    const int kbytes = jb.K * ESZ;
    const int nk = (kbytes + UM_KB - 1) / UM_KB;
    const uint32_t idesc = umma_idesc(KIND == 0 ? 2 : 1);
    bool ok = true;
    uint32_t phase[UM_STAGES] = {0u, 0u};

    auto issue_loads = [&](int kc, int s) {
        const uint32_t st = sbase + s * stage_bytes;
        for (int p = 0; p < P; ++p) {
            load_tile<ESZ>(st + p * 16384u, (const unsigned char*)jb.A[p] + (int64_t)m0 * jb.lda * ESZ,
                           jb.M - m0, kc * UM_KB, kbytes, (int64_t)jb.lda * ESZ);
            load_tile<ESZ>(st + (P + p) * 16384u, (const unsigned char*)jb.B[p] + (int64_t)n0 * jb.ldb * ESZ,
                           jb.N - n0, kc * UM_KB, kbytes, (int64_t)jb.ldb * ESZ);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };

    issue_loads(0, 0);
    for (int kc = 0; kc < nk && ok; ++kc) {
        const int s = kc & 1;
        if (kc + 1 < nk) {
            const int s1 = s ^ 1;
            if (kc >= 1) {  // MMAs of chunk kc-1 read stage s1: wait for their commit
                ok = __syncthreads_and(mbar_wait(&bar[s1], phase[s1]) ? 1 : 0) != 0;
                phase[s1] ^= 1u;
                if (!ok) break;
            }
            issue_loads(kc + 1, s1);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        // make this thread's cp.async data visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t st = sbase + s * stage_bytes;
            for (int p = 0; p < P; ++p) {
                const uint64_t da = umma_desc(st + p * 16384u);
                const uint64_t db = umma_desc(st + (P + p) * 16384u);
#pragma unroll
                for (int kk = 0; kk < UM_KB / 32; ++kk) {  // 32 bytes of K per instruction
                    const uint32_t acc = (kc > 0 || p > 0 || kk > 0) ? 1u : 0u;
                    const uint64_t adv = (uint64_t)((kk * 32) >> 4);
                    if (KIND == 0)
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                            "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(acc)
                            : "memory");
                    else
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                            "l"(da + adv), "l"(db + adv), "r"(idesc), "r"(acc)
                            : "memory");
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[s]))
                         : "memory");
        }
    }
    // wait for the last commit (covers every earlier MMA)
    if (ok && nk > 0) {
        const int s = (nk - 1) & 1;
        ok = __syncthreads_and(mbar_wait(&bar[s], phase[s]) ? 1 : 0) != 0;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows m0 + 32w + lane), 32 columns at a time
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < UM_TILE; c0 += 32) {
            uint32_t v[32];
            const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]),
                  "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]),
                  "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                : "r"(ta));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < jb.M) {
                float* out = jb.C + (int64_t)row * jb.ldc + n0 + c0;
#pragma unroll
                for (int q = 0; q < 32; ++q)
                    if (n0 + c0 + q < jb.N) out[q] = __uint_as_float(v[q]);
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

// ------------------------------------------------------------------ split-TF32, warp-specialized
// C = A1 B1^T + A1 B2^T + A2 B1^T for pre-tiled operands (layout in mmf_internal.h).  One CTA per
// 128 x BN tile of C (BN = 128 or 256; the wider tile reads A once per 256 columns of C).  Warps:
// one producer (one lane) streams the operand tiles of each K step (A1, A2: 16 KB each; B1, B2:
// BN/128 adjacent 16-KB tiles each) into a ring of stages (3, or 2 for BN = 256) with
// cp.async.bulk (completion counted on full[stage]); one MMA warp (one lane) issues the 12
// tcgen05.mma of the step (M = 128, N = BN) and frees the stage with tcgen05.commit on
// empty[stage]; BN / 32 epilogue warps, two per TMEM lane quadrant for BN = 256, each own 32 rows
// and 128 columns of the tile.
// The tensor cores' FP32 accumulation loses accuracy over long K, so the sum is cut into chunks
// of TF_KC K steps: each chunk is accumulated in one of two TMEM buffers (commit on accfull[b])
// and added, rounded to nearest, into the epilogue warps' registers, which then free the buffer
// (accempty[b]) while the next chunk runs.  Every wait is bounded and ends on a shared abort flag.
#define TF_TILE_BYTES 16384u
#define TF_KC 4

__device__ __forceinline__ bool tf_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
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

__device__ __forceinline__ void tf_ld32(uint32_t ta, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
          "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
          "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
}

template <int BN>
__global__ void __launch_bounds__(32 * (BN / 32 + 2), 1) k_tf3_gemm(const Tf3Job* __restrict__ jobs,
                                                                   int* __restrict__ err) {
    constexpr int NE = BN / 32;              // epilogue warps (two per TMEM lane quadrant for BN = 256)
    constexpr int NST = BN == 128 ? 3 : 2;   // pipeline stages
    constexpr uint32_t BT = (uint32_t)(BN / 128) * TF_TILE_BYTES;  // one piece of the B tile
    constexpr uint32_t SB = 2u * TF_TILE_BYTES + 2u * BT;         // stage bytes
    extern __shared__ __align__(1024) unsigned char tf_smem[];
    __shared__ uint64_t full[NST], empty[NST], accfull[2], accempty[2];
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    const Tf3Job jb = jobs[blockIdx.z];
    const int I = blockIdx.x, J = blockIdx.y;
    if (I * 128 >= jb.M || J * BN >= jb.N) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)tf_smem + 1023) & ~(uintptr_t)1023);
    const uint32_t sbase = smem_u32(base);
    volatile int* abort_flag = &abort_s;
    if (threadIdx.x == 0) {
        abort_s = 0;
        for (int q = 0; q < NST; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], 1);
        }
        for (int q = 0; q < 2; ++q) {
            mbar_init(&accfull[q], 1);
            mbar_init(&accempty[q], NE);  // one arrival per epilogue warp
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(2u * BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int nt = tf3_nt(jb.K), nqa = tf3_nq(jb.M), nqb = tf3_nq(jb.N);
    const int nch = (nt + TF_KC - 1) / TF_KC;
    const int64_t pa = tf3_piece(jb.M, jb.K), pb = tf3_piece(jb.N, jb.K);

    if (warp == NE) {
        if (lane == 0) {
            // B row tiles of this CTA present in the operand (the last one may hold one of two)
            const int jt0 = J * (BN / 128), nbv = min(BN / 128, nqb - jt0);
            const uint32_t bbytes = (uint32_t)nbv * TF_TILE_BYTES;
            for (int t = 0; t < nt; ++t) {
                const int st = t % NST;
                const uint32_t use = (uint32_t)(t / NST);
                if (use > 0 && !tf_wait(&empty[st], (use - 1) & 1u, abort_flag)) break;
                const uint32_t fb = smem_u32(&full[st]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb),
                             "r"(2u * TF_TILE_BYTES + 2u * bbytes)
                             : "memory");
                const uint32_t dst = sbase + (uint32_t)st * SB;
                const float* src[4] = {jb.A + ((int64_t)t * nqa + I) * 4096, jb.A + pa + ((int64_t)t * nqa + I) * 4096,
                                       jb.B + ((int64_t)t * nqb + jt0) * 4096, jb.B + pb + ((int64_t)t * nqb + jt0) * 4096};
                const uint32_t off[4] = {0u, TF_TILE_BYTES, 2u * TF_TILE_BYTES, 2u * TF_TILE_BYTES + BT};
                const uint32_t len[4] = {TF_TILE_BYTES, TF_TILE_BYTES, bbytes, bbytes};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            dst + off[q]),
                        "l"(src[q]), "r"(len[q]), "r"(fb)
                        : "memory");
            }
        }
    } else if (warp == NE + 1) {
        if (lane == 0) {
            const uint32_t idesc = umma_idesc_mn(2, 128u, (uint32_t)BN);  // TF32, M = 128, N = BN
            for (int t = 0; t < nt; ++t) {
                const int st = t % NST;
                const int ch = t / TF_KC, kin = t - ch * TF_KC, bsel = ch & 1;
                if (kin == 0 && ch >= 2 && !tf_wait(&accempty[bsel], (uint32_t)((ch >> 1) - 1) & 1u, abort_flag)) break;
                if (!tf_wait(&full[st], (uint32_t)(t / NST) & 1u, abort_flag)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t sa = sbase + (uint32_t)st * SB;
                const uint64_t a1 = umma_desc(sa), a2 = umma_desc(sa + TF_TILE_BYTES);
                const uint64_t b1 = umma_desc(sa + 2 * TF_TILE_BYTES), b2 = umma_desc(sa + 2 * TF_TILE_BYTES + BT);
                const uint32_t dacc = tmem + (uint32_t)(bsel * BN);
#pragma unroll
                for (int q = 0; q < 4; ++q) {  // 32 bytes (8 TF32) of K per instruction
                    const uint64_t adv = (uint64_t)((q * 32) >> 4);
                    const uint32_t acc0 = (kin > 0 || q > 0) ? 1u : 0u;
                    const uint64_t pa_[3] = {a1, a1, a2}, pb_[3] = {b1, b2, b1};
#pragma unroll
                    for (int pp = 0; pp < 3; ++pp) {
                        const uint32_t accf = (pp > 0) ? 1u : acc0;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
                            "l"(pa_[pp] + adv), "l"(pb_[pp] + adv), "r"(idesc), "r"(accf)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[st]))
                             : "memory");
                if (kin == TF_KC - 1 || t == nt - 1)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&accfull[bsel]))
                                 : "memory");
            }
        }
    } else {
        // epilogue: warp w holds rows 32 (w % 4) .. +31 of the tile (its TMEM lanes) and columns
        // 128 (w / 4) .. +127; the chunks are summed in registers
        float acc[128];
#pragma unroll
        for (int q = 0; q < 128; ++q) acc[q] = 0.f;
        bool ok = true;
        for (int ch = 0; ch < nch && ok; ++ch) {
            const int bsel = ch & 1;
            if (!tf_wait(&accfull[bsel], (uint32_t)(ch >> 1) & 1u, abort_flag)) { ok = false; break; }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int c0 = 0; c0 < 128; c0 += 32) {
                uint32_t v[32];
                tf_ld32(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(bsel * BN + (warp >> 2) * 128 + c0), v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) acc[c0 + q] += __uint_as_float(v[q]);
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[bsel])) : "memory");
            }
        }
        if (ok) {
            const int row = I * 128 + (warp & 3) * 32 + lane;
#pragma unroll
            for (int c0 = 0; c0 < 128; c0 += 32) {
                const int col = J * BN + (warp >> 2) * 128 + c0;
                if (col >= jb.N) break;
                if (jb.mode == TF3_OPERAND) {
                    // the row's 32 values are one 128-byte row of K-tile col / 32 (16-byte chunks
                    // swizzled); rows past M are written as zeros
                    const int64_t pc = tf3_piece(jb.M, jb.N);
                    const int sw = row & 7;
                    // start of the row: tf3_pos of column col (a multiple of 32) holds chunk 0 at
                    // its swizzled place sw
                    float* o1 = jb.C + tf3_pos(jb.M, jb.N, 0, row, col) - (sw << 2);
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        float4 h = make_float4(0.f, 0.f, 0.f, 0.f), l = h;
                        if (row < jb.M) {
                            const float x0 = acc[c0 + 4 * q], x1 = acc[c0 + 4 * q + 1];
                            const float x2 = acc[c0 + 4 * q + 2], x3 = acc[c0 + 4 * q + 3];
                            h = make_float4(tf32_round(x0), tf32_round(x1), tf32_round(x2), tf32_round(x3));
                            l = make_float4(tf32_round(x0 - h.x), tf32_round(x1 - h.y), tf32_round(x2 - h.z),
                                            tf32_round(x3 - h.w));
                        }
                        *reinterpret_cast<float4*>(o1 + ((q ^ sw) << 2)) = h;
                        *reinterpret_cast<float4*>(o1 + pc + ((q ^ sw) << 2)) = l;
                    }
                } else if (row < jb.M) {
                    float* out = jb.C + (int64_t)row * jb.ldc + col;
                    if (jb.mode == TF3_SUBTRACT) {
                        // C is 16-byte aligned per row and N is even
#pragma unroll
                        for (int q = 0; q < 32; q += 4) {
                            if (col + q + 3 < jb.N) {
                                float4 c = *reinterpret_cast<float4*>(out + q);
                                c.x -= acc[c0 + q];
                                c.y -= acc[c0 + q + 1];
                                c.z -= acc[c0 + q + 2];
                                c.w -= acc[c0 + q + 3];
                                *reinterpret_cast<float4*>(out + q) = c;
                            } else {
#pragma unroll
                                for (int u = 0; u < 4; ++u)
                                    if (col + q + u < jb.N) out[q + u] -= acc[c0 + q + u];
                            }
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < 32; ++q)
                            if (col + q < jb.N) out[q] = acc[c0 + q];
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && abort_s) atomicExch(err, 1);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2u * BN) : "memory");
}

template <int BN>
static cudaError_t launch_tf3(const void* jobs, int count, int Mmax, int Nmax, int* err, cudaStream_t stream) {
    constexpr int NST = BN == 128 ? 3 : 2;
    const size_t sm = (size_t)NST * (2 * TF_TILE_BYTES + 2 * (BN / 128) * TF_TILE_BYTES) + 1024;
    cudaError_t e = cudaFuncSetAttribute(k_tf3_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    dim3 grid((Mmax + 127) / 128, (Nmax + BN - 1) / BN, count);
    k_tf3_gemm<BN><<<grid, 32 * (BN / 32 + 2), sm, stream>>>((const Tf3Job*)jobs, err);
    return cudaGetLastError();
}

// 256-wide tiles (A read once per 256 columns of C) wherever the widest product allows
cudaError_t mmf_launch_tf3(const void* jobs, int count, int Mmax, int Nmax, int* err, cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    return Nmax >= 256 ? launch_tf3<256>(jobs, count, Mmax, Nmax, err, stream)
                       : launch_tf3<128>(jobs, count, Mmax, Nmax, err, stream);
}

// jobs: device array of `count` UmmaJob; grid covers the largest M and N among them
cudaError_t mmf_launch_umma(const void* jobs, int count, int P, int Mmax, int Nmax, int kind, int* err,
                            cudaStream_t stream) {
    if (count <= 0) return cudaSuccess;
    if (P < 1 || P > UM_MAXP) return cudaErrorInvalidValue;
    const size_t sm = (size_t)UM_STAGES * 2 * P * 16384 + 1024;
    dim3 grid((Mmax + UM_TILE - 1) / UM_TILE, (Nmax + UM_TILE - 1) / UM_TILE, count);
    cudaError_t e;
    if (kind == 0) {
        e = cudaFuncSetAttribute(k_umma_gemm<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_umma_gemm<0><<<grid, UM_THREADS, sm, stream>>>((const UmmaJob*)jobs, P, err);
    } else {
        e = cudaFuncSetAttribute(k_umma_gemm<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_umma_gemm<1><<<grid, UM_THREADS, sm, stream>>>((const UmmaJob*)jobs, P, err);
    }
    return cudaGetLastError();
}

size_t mmf_umma_job_bytes() { return sizeof(UmmaJob); }

// ------------------------------------------------------------------ self-test
// The engine against a plain FP32 reference on seeded data (TF32-exact or BF16-exact inputs, so
// both sides compute exact products and differ only by summation order).
__global__ void k_umma_fill(float* A, int rows, int K, int ld, uint32_t seed, int kind, uint16_t* A16) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)rows * K;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / K), k = (int)(e % K);
        uint32_t x = (uint32_t)e * 2654435761u ^ seed;
        x ^= x >> 13; x *= 0x5bd1e995u; x ^= x >> 15;
        float v = ((int)(x & 0xFFF) - 2048) / 256.0f;  // 12-bit values: exact in TF32 and (mostly) BF16
        if (kind == 1) v = __bfloat162float(__float2bfloat16_rn(v));
        A[(int64_t)r * ld + k] = v;
        if (A16) A16[(int64_t)r * ld + k] = __bfloat16_as_ushort(__float2bfloat16_rn(v));
    }
}
__global__ void k_umma_ref(const float* A, const float* B, double* C, int M, int N, int K, int lda, int ldb) {
    const int m = blockIdx.y, n = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M || n >= N) return;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += (double)A[(int64_t)m * lda + k] * (double)B[(int64_t)n * ldb + k];
    C[(int64_t)m * N + n] = acc;
}
__global__ void k_umma_cmp(const float* C, const double* R, int64_t tot, double scale, double* out) {
    double mx = 0.0, ref = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        mx = fmax(mx, fabs((double)C[e] - scale * R[e]));
        ref = fmax(ref, fabs(scale * R[e]));
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

int mmf_umma_selftest_impl(int M, int N, int K, int kind, int P, double* max_abs, double* max_ref) {
    if (M < 1 || N < 1 || K < 1 || P < 1 || P > UM_MAXP || (kind != 0 && kind != 1)) return -1;
    const int align = kind == 0 ? 4 : 8;
    const int ld = (K + align - 1) / align * align;
    float *A = nullptr, *B = nullptr, *C = nullptr;
    uint16_t *A16 = nullptr, *B16 = nullptr;
    double *R = nullptr, *out = nullptr;
    UmmaJob* dj = nullptr;
    int* err = nullptr;
    int rc = 0;
    cudaError_t e = cudaMalloc(&A, sizeof(float) * (size_t)M * ld);
    if (e == cudaSuccess) e = cudaMalloc(&B, sizeof(float) * (size_t)N * ld);
    if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&A16, sizeof(uint16_t) * (size_t)M * ld);
    if (e == cudaSuccess) e = cudaMalloc(&B16, sizeof(uint16_t) * (size_t)N * ld);
    if (e == cudaSuccess) e = cudaMalloc(&R, sizeof(double) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dj, sizeof(UmmaJob));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(out, 0, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(A, 0, sizeof(float) * (size_t)M * ld);
    if (e == cudaSuccess) e = cudaMemset(B, 0, sizeof(float) * (size_t)N * ld);
    if (e == cudaSuccess) {
        k_umma_fill<<<256, 256>>>(A, M, K, ld, 12345u, kind, A16);
        k_umma_fill<<<256, 256>>>(B, N, K, ld, 777u, kind, B16);
        UmmaJob j;
        memset(&j, 0, sizeof(j));
        for (int p = 0; p < P; ++p) {  // the same product P times: C = P * A B^T
            j.A[p] = kind == 0 ? (const void*)A : (const void*)A16;
            j.B[p] = kind == 0 ? (const void*)B : (const void*)B16;
        }
        j.C = C;
        j.M = M; j.N = N; j.K = K; j.lda = ld; j.ldb = ld; j.ldc = N;
        e = cudaMemcpy(dj, &j, sizeof(j), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = mmf_launch_umma(dj, 1, P, M, N, kind, err, 0);
    if (e == cudaSuccess) {
        k_umma_ref<<<dim3((N + 127) / 128, M), 128>>>(A, B, R, M, N, K, ld, ld);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {  // the engine summed the same product P times
        k_umma_cmp<<<256, 256>>>(C, R, (int64_t)M * N, (double)P, out);
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
    cudaFree(A); cudaFree(B); cudaFree(C); cudaFree(A16); cudaFree(B16); cudaFree(R); cudaFree(out);
    cudaFree(dj); cudaFree(err);
    return rc;
}

// ------------------------------------------------------------------ split-TF32 engine self-test
// k_tf3_gemm on seeded FP32 operands that are not TF32-exact (24-bit mantissas), in each output
// mode, against an FP64 reference; the error of a sequential FP32 dot product (fmaf, round to
// nearest) is reported beside it.  Errors are relative to sum_k |a_k b_k| of each entry.
__global__ void k_tf3_fill(float* A, int64_t count, uint32_t seed) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)e * 2654435761u ^ seed;
        x ^= x >> 13; x *= 0x5bd1e995u; x ^= x >> 15; x *= 0x27d4eb2fu; x ^= x >> 16;
        A[e] = (float)((int)(x >> 8) - (1 << 23)) / (float)(1 << 23);  // 24-bit values in [-1, 1)
    }
}
__global__ void k_tf3_tile(const float* __restrict__ A, int rows, int K, float* __restrict__ P) {
    const int64_t tot = (int64_t)tf3_nq(rows) * 128 * tf3_nt(K) * 32;
    const int Kp = tf3_nt(K) * 32;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(e / Kp), k = (int)(e - (int64_t)r * Kp);
        const float v = (r < rows && k < K) ? A[(int64_t)r * K + k] : 0.f;
        const float h = tf32_round(v);
        P[tf3_pos(rows, K, 0, r, k)] = h;
        P[tf3_pos(rows, K, 1, r, k)] = tf32_round(v - h);
    }
}
__global__ void k_tf3_ref(const float* __restrict__ A, const float* __restrict__ B, int M, int N, int K,
                          double* __restrict__ R, double* __restrict__ S, float* __restrict__ R32) {
    const int m = blockIdx.y, n = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M || n >= N) return;
    double acc = 0.0, sc = 0.0;
    float a32 = 0.f;
    for (int k = 0; k < K; ++k) {
        const float a = A[(int64_t)m * K + k], b = B[(int64_t)n * K + k];
        acc += (double)a * (double)b;
        sc += fabs((double)a * (double)b);
        a32 = fmaf(a, b, a32);
    }
    R[(int64_t)m * N + n] = acc;
    S[(int64_t)m * N + n] = sc;
    R32[(int64_t)m * N + n] = a32;
}
__global__ void k_tf3_cmp(const float* __restrict__ C, const float* __restrict__ C0, const double* __restrict__ R,
                          const double* __restrict__ S, const float* __restrict__ R32, int M, int N, int mode,
                          double* out) {
    double mx = 0.0, mx32 = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)M * N;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int m = (int)(e / N), n = (int)(e - (int64_t)m * N);
        double c, x = R[e];
        if (mode == TF3_OPERAND) {
            c = (double)C[tf3_pos(M, N, 0, m, n)] + (double)C[tf3_pos(M, N, 1, m, n)];
        } else {
            c = C[e];
            if (mode == TF3_SUBTRACT) x = (double)C0[e] - x;
        }
        const double sc = fmax(S[e], 1e-300);
        mx = fmax(mx, fabs(c - x) / sc);
        mx32 = fmax(mx32, fabs((double)R32[e] - R[e]) / sc);
    }
    for (int o = 16; o > 0; o >>= 1) {
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        mx32 = fmax(mx32, __shfl_xor_sync(0xffffffffu, mx32, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax((unsigned long long*)&out[0], __double_as_longlong(mx));
        atomicMax((unsigned long long*)&out[1], __double_as_longlong(mx32));
    }
}

int mmf_tf3_selftest_impl(int M, int N, int K, int mode, double* max_rel, double* max_rel_fp32) {
    if (M < 1 || M > 65535 || N < 1 || K < 1 || mode < 0 || mode > 2 || (mode == TF3_OPERAND && N % 32 != 0))
        return -1;
    if ((int64_t)M * K > (1 << 26) || (int64_t)N * K > (1 << 26) || (int64_t)M * N > (1 << 26)) return -1;
    float *A = nullptr, *B = nullptr, *PA = nullptr, *PB = nullptr, *C = nullptr, *C0 = nullptr, *R32 = nullptr;
    double *R = nullptr, *S = nullptr, *out = nullptr;
    Tf3Job* dj = nullptr;
    int* err = nullptr;
    const int64_t pa = tf3_piece(M, K), pb = tf3_piece(N, K);
    const int64_t nc = mode == TF3_OPERAND ? 2 * tf3_piece(M, N) : (int64_t)M * N;
    cudaError_t e = cudaMalloc(&A, sizeof(float) * (size_t)M * K);
    if (e == cudaSuccess) e = cudaMalloc(&B, sizeof(float) * (size_t)N * K);
    if (e == cudaSuccess) e = cudaMalloc(&PA, sizeof(float) * 2 * (size_t)pa);
    if (e == cudaSuccess) e = cudaMalloc(&PB, sizeof(float) * 2 * (size_t)pb);
    if (e == cudaSuccess) e = cudaMalloc(&C, sizeof(float) * (size_t)nc);
    if (e == cudaSuccess) e = cudaMalloc(&C0, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&R32, sizeof(float) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&R, sizeof(double) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&S, sizeof(double) * (size_t)M * N);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMalloc(&dj, sizeof(Tf3Job));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(out, 0, sizeof(double) * 2);
    if (e == cudaSuccess) e = cudaMemset(err, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_tf3_fill<<<256, 256>>>(A, (int64_t)M * K, 12345u);
        k_tf3_fill<<<256, 256>>>(B, (int64_t)N * K, 777u);
        k_tf3_fill<<<256, 256>>>(C0, (int64_t)M * N, 4242u);
        k_tf3_tile<<<512, 256>>>(A, M, K, PA);
        k_tf3_tile<<<512, 256>>>(B, N, K, PB);
        if (mode == TF3_OPERAND) e = cudaMemset(C, 0xff, sizeof(float) * (size_t)nc);  // padding must be rewritten
        else e = cudaMemcpy(C, C0, sizeof(float) * (size_t)M * N, cudaMemcpyDeviceToDevice);
    }
    if (e == cudaSuccess) {
        Tf3Job j;
        j.A = PA; j.B = PB; j.C = C;
        j.M = M; j.N = N; j.K = K; j.ldc = N; j.mode = mode;
        e = cudaMemcpy(dj, &j, sizeof(j), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = mmf_launch_tf3(dj, 1, M, N, err, 0);
    if (e == cudaSuccess) {
        k_tf3_ref<<<dim3((N + 127) / 128, M), 128>>>(A, B, M, N, K, R, S, R32);
        k_tf3_cmp<<<256, 256>>>(C, C0, R, S, R32, M, N, mode, out);
        e = cudaDeviceSynchronize();
    }
    double hout[2] = {0, 0};
    int herr = 0;
    if (e == cudaSuccess) e = cudaMemcpy(hout, out, sizeof(hout), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost);
    int rc = 0;
    if (e != cudaSuccess) rc = -4;
    else if (herr) rc = 1;
    *max_rel = hout[0];
    *max_rel_fp32 = hout[1];
    cudaFree(A); cudaFree(B); cudaFree(PA); cudaFree(PB); cudaFree(C); cudaFree(C0); cudaFree(R32);
    cudaFree(R); cudaFree(S); cudaFree(out); cudaFree(dj); cudaFree(err);
    return rc;
}
