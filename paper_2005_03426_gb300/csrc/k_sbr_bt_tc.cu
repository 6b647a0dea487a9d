// k_sbr_bt_tc.cu -- S5 of the band path on the tensor cores (mixed path, half-bandwidth 33..64):
// Z = Q Y with Q = prod_j prod_s H(j, s) the bulge chase's reflectors (Sec. 3.2's eigenvectors of
// H_F from those of the tridiagonal matrix).
//
// The reflectors are applied in the chase's valid order, pass s ascending and within a pass sweep
// j descending (k_sbr.cu).  Within pass s the reflectors of 64 consecutive sweeps
// jlo .. jhi (jhi = n - 2 - s b - 64 g for block g = 0, 1, ...) are applied as one block:
//     H(jlo) H(jlo + 1) ... H(jhi) = I - V T V^H            (compact WY, Schreiber & Van Loan 1989)
// where column c of V is v_{jlo+c} placed at its rows, V(i, c) = v_{jlo+c}[i - c] for
// 0 <= i - c < b (a staircase of 64 + b - 1 <= 127 rows starting at row R0 = jlo + 1 + s b), and T
// is upper triangular, T(c, c) = tau_c, T(0:c, c) = -tau_c T(0:c, 0:c) V(:, 0:c)^H v_c.
// Consecutive blocks of a pass share b - 1 rows, so blocks apply in sequence.
//
// k_sbr_wy, one CTA per block (blocks are independent): T, then Y = V T, and both products'
// B operands in split-TF32 pieces and the tensor cores' shared-memory layout, into the system's
// operand area (512 KB per block).  k_sbr_bt_tc, one CTA per (system, 128 columns of Z): Z's
// columns are independent, and the CTA applies every block of every pass to its slab as two
// split-TF32 products on the tcgen05 engine (FP32 operands cut into two TF32 pieces x = x1 + x2,
// products x1 y1 + x1 y2 + x2 y1):
//     (1)  W^T = Z_R^T conj(V)       128 x 64 complex, K = the window's 128 rows
//     (2)  Z_R^T -= W^T Y^T          128 x 128,        K = 64         (Y = V T)
// Complex products are real products with K' = 2K interleaved (Re, Im) entries per row: an A row
// [ar_0, ai_0, ar_1, ai_1, ...] against B rows, two per complex output column, chosen so that the
// output's columns 2m and 2m + 1 hold its real and imaginary parts:
//     (1)  B'(2j) = [Vr(i,j), Vi(i,j)]_i     B'(2j+1) = [-Vi(i,j), Vr(i,j)]_i
//     (2)  B'(2i) = [Yr(i,j), -Yi(i,j)]_j    B'(2i+1) = [Yi(i,j), Yr(i,j)]_j
// so that product (1)'s accumulator, read back row by row, is product (2)'s A operand in that
// interleaved order.  TMEM (512 columns): (1) in two accumulators of four K chunks each (columns
// 256 and 384), (2) over 256 columns at 0.  Per K chunk (32 real entries) one thread starts the
// bulk copies (cp.async.bulk, completion counted on the stage's full barrier) of the chunk's B
// pieces while the CTA's threads build the A pieces (Z's window, or product (1)'s accumulator)
// into the same 96 KB stage; one thread then issues the chunk's tcgen05.mma and commits them to
// the stage's free barrier, so that the next chunk is loaded and built while they run.  The
// epilogue subtracts (2) from Z, which stays row-major in global memory (the slab's 128-row
// window is L2-resident; each pass reads and writes it once).  Every wait is bounded; one that
// gives up sets the system's status to MMF_ST_NOCONV and the CTA stops.
#include "mmf_internal.h"
#include "umma_common.h"

#define SBT_NB 64                 // sweeps per block
#define SBT_THREADS 256
#define SBT_STAGE 98304u          // A: 2 x 16 KB, B: 2 x 32 KB (N up to 256)
#define SBT_TMEM_COLS 512u
#define SBT_WY_SMEM ((3 * 64 * 65 + 64) * 8)
// one block's operands in the operand area (floats): product (1)'s B, 8 chunks x 2 pieces x
// 128 x 32, then product (2)'s B, 4 chunks x 2 pieces x 256 x 32
#define SBT_B1_FLOATS (8 * 2 * 4096)
#define SBT_OPS_FLOATS (SBT_B1_FLOATS + 4 * 2 * 8192)

// blocks of pass s: sweeps 0 .. n-2-s b in groups of 64 from the top
__host__ __device__ __forceinline__ int sbt_nblk(int n, int b, int s) { return (n - 1 - s * b + SBT_NB - 1) / SBT_NB; }
__host__ __device__ inline int64_t sbt_blocks(int n, int b) {
    int64_t t = 0;
    for (int s = 0; s < sbr_passes(n, b); ++s) t += sbt_nblk(n, b, s);
    return t;
}
// operand-area size (BF16 units, the area's unit) of a system's blocks
int64_t mmf_sbt_ops_elems(int n, int b) { return 2 * sbt_blocks(n, b) * (int64_t)SBT_OPS_FLOATS; }
__device__ __forceinline__ float* sbt_ops(void* pool, const MmfDesc& d) {
    return reinterpret_cast<float*>(reinterpret_cast<uint16_t*>(pool) + d.oz_off);
}
__device__ __forceinline__ int sbt_swz(int r, int kq) {  // float offset of row r's 16-byte chunk kq
    return (r >> 3) * 256 + (r & 7) * 32 + ((kq ^ (r & 7)) << 2);
}
__device__ __forceinline__ void sbt_put4(float* hi, float* lo, int off, float x0, float x1, float x2, float x3) {
    const float4 h = make_float4(tf32_round(x0), tf32_round(x1), tf32_round(x2), tf32_round(x3));
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) =
        make_float4(tf32_round(x0 - h.x), tf32_round(x1 - h.y), tf32_round(x2 - h.z), tf32_round(x3 - h.w));
}

// ------------------------------------------------------------------ per-block operands
// One CTA per block: V's 64 columns (v_c[t], zero past b and past the block's sweeps), the Gram
// entries G(m, c) = v_m^H v_c of the staircase (nonzero for 0 < c - m < b), T, then both
// products' B operands (FP32 arithmetic: the products that use them
// have FP32 accuracy): (1) from V(i, j) = Vs[j][i - j], (2) from Y(i, j) = sum_{k <= j} V(i, k)
// T(k, j).  Each thread writes float4 groups (four consecutive K' entries of one row) of both
// pieces at their swizzled places.
__global__ void __launch_bounds__(256) k_sbr_wy(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                               const double2* __restrict__ store_base, void* __restrict__ pool) {
    extern __shared__ float2 wy_sm[];  // Vs, Gs, Ts: 64 x 65 each; tau: 64
    float2(*Vs)[65] = reinterpret_cast<float2(*)[65]>(wy_sm);
    float2(*Gs)[65] = reinterpret_cast<float2(*)[65]>(wy_sm + 64 * 65);
    float2(*Ts)[65] = reinterpret_cast<float2(*)[65]>(wy_sm + 2 * 64 * 65);
    float2* tau_s = wy_sm + 3 * 64 * 65;
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, b = d.band;
    int g = blockIdx.x, s = 0;
    const int np = sbr_passes(n, b);
    int64_t pre = 0;  // blocks before this one in the system's operand area
    for (; s < np; ++s) {
        const int nb = sbt_nblk(n, b, s);
        if (g < nb) break;
        g -= nb;
        pre += nb;
    }
    if (s >= np) return;
    const int jtop = n - 2 - s * b, jhi = jtop - SBT_NB * g, jlo = max(0, jhi - (SBT_NB - 1));
    const int nbk = jhi - jlo + 1;
    const int64_t off = sbr_off(n, b, s);
    const float2* V = reinterpret_cast<const float2*>(store_base + d.mat_off);
    const float2* Tau = V + sbr_nref(n, b) * b;
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * 64; e += 256) {
        const int c = e >> 6, t = e & 63;
        Vs[c][t] = (c < nbk && t < b) ? V[(off + jlo + c) * b + t] : make_float2(0.f, 0.f);
        Ts[c][t] = make_float2(0.f, 0.f);
    }
    if (tid < 64) tau_s[tid] = tid < nbk ? Tau[off + jlo + tid] : make_float2(0.f, 0.f);
    __syncthreads();
    // G(m, c) for m < c: sum_t conj(v_m[t + c - m]) v_c[t], t + c - m < b
    for (int e = tid; e < 64 * 64; e += 256) {
        const int m = e & 63, c = e >> 6, dlt = c - m;
        float gr = 0.f, gi = 0.f;
        if (dlt > 0 && dlt < b)
            for (int t = 0; t + dlt < b; ++t) {
                const float2 a = Vs[m][t + dlt], v = Vs[c][t];
                gr = fmaf(a.x, v.x, fmaf(a.y, v.y, gr));
                gi = fmaf(a.x, v.y, fmaf(-a.y, v.x, gi));
            }
        Gs[m][c] = make_float2(gr, gi);
    }
    __syncthreads();
    // T by merging compact-WY factors of adjacent groups (1, 2, 4, ... 32 columns): for groups A
    // (columns a .. a+h-1) and B (a+h .. a+2h-1), the product of their reflectors has
    //     T = [[T_A, -T_A G_AB T_B], [0, T_B]],   G_AB = V_A^H V_B,
    // which is the column recurrence taken h columns at a time (it holds for any tau, including
    // the zeros of the block's missing sweeps).  P = G_AB T_B goes to T's free lower triangle
    // (P(i, j) at Ts[j][i], i < j) between the two steps.
    if (tid < 64) Ts[tid][tid] = tau_s[tid];
    __syncthreads();
    for (int h = 1; h < 64; h *= 2) {
        for (int e = tid; e < 32 * h; e += 256) {  // (64 / 2h) group pairs x h x h entries
            const int pr = e / (h * h), rem = e - pr * h * h, ii = rem / h, jj = rem - ii * h;
            const int a = 2 * h * pr, i = a + ii, j = a + h + jj;
            float pr_ = 0.f, pi_ = 0.f;
            for (int m = a + h; m <= j; ++m) {  // T_B upper triangular
                const float2 gg = Gs[i][m], t = Ts[m][j];
                pr_ = fmaf(gg.x, t.x, fmaf(-gg.y, t.y, pr_));
                pi_ = fmaf(gg.x, t.y, fmaf(gg.y, t.x, pi_));
            }
            Ts[j][i] = make_float2(pr_, pi_);
        }
        __syncthreads();
        for (int e = tid; e < 32 * h; e += 256) {
            const int pr = e / (h * h), rem = e - pr * h * h, ii = rem / h, jj = rem - ii * h;
            const int a = 2 * h * pr, i = a + ii, j = a + h + jj;
            float tr = 0.f, ti = 0.f;
            for (int l = i; l < a + h; ++l) {  // T_A upper triangular
                const float2 t = Ts[i][l], pp = Ts[j][l];
                tr = fmaf(t.x, pp.x, fmaf(-t.y, pp.y, tr));
                ti = fmaf(t.x, pp.y, fmaf(t.y, pp.x, ti));
            }
            Ts[i][j] = make_float2(-tr, -ti);
        }
        __syncthreads();
    }
    float* ops = sbt_ops(pool, d) + (pre + g) * (int64_t)SBT_OPS_FLOATS;
    // (1): rows 2j (Re) and 2j + 1 (Im) of output column j; K' 4-groups (i, i + 1) of chunk q
    // (eight consecutive threads fill the eight 16-byte groups of one row: one 128-byte line)
    for (int e = tid; e < 64 * 64; e += 256) {
        const int kq = e & 7, j = (e >> 3) & 63, q = e >> 9, i = 16 * q + 2 * kq;  // rows i, i + 1
        const float2 v0 = (i - j >= 0 && i - j < 64) ? Vs[j][i - j] : make_float2(0.f, 0.f);
        const float2 v1 = (i + 1 - j >= 0 && i + 1 - j < 64) ? Vs[j][i + 1 - j] : make_float2(0.f, 0.f);
        float* hi = ops + (int64_t)(2 * q) * 4096;
        float* lo = hi + 4096;
        sbt_put4(hi, lo, sbt_swz(2 * j, kq), v0.x, v0.y, v1.x, v1.y);
        sbt_put4(hi, lo, sbt_swz(2 * j + 1, kq), -v0.y, v0.x, -v1.y, v1.x);
    }
    // (2): Y(i, j) for the pair j, j + 1; rows 2i (Re) and 2i + 1 (Im) of window row i
    for (int e = tid; e < 128 * 32; e += 256) {
        const int kq = e & 7, i = (e >> 3) & 127, q = e >> 10, j = 16 * q + 2 * kq;
        // Y(i, j) and Y(i, j + 1) in one pass over k (V(i, k) = 0 unless 0 <= i - k < 64; T upper
        // triangular, so T(k, j) is used for k <= j only: its lower part holds scratch)
        float yr0 = 0.f, yi0 = 0.f, yr1 = 0.f, yi1 = 0.f;
        const int khi = min(j + 1, i);
        for (int k = max(0, i - 63); k <= khi; ++k) {
            const float2 v = Vs[k][i - k], t1 = Ts[k][j + 1];
            const float2 t0 = k <= j ? Ts[k][j] : make_float2(0.f, 0.f);
            yr0 = fmaf(v.x, t0.x, fmaf(-v.y, t0.y, yr0));
            yi0 = fmaf(v.x, t0.y, fmaf(v.y, t0.x, yi0));
            yr1 = fmaf(v.x, t1.x, fmaf(-v.y, t1.y, yr1));
            yi1 = fmaf(v.x, t1.y, fmaf(v.y, t1.x, yi1));
        }
        const float2 y[2] = {make_float2(yr0, yi0), make_float2(yr1, yi1)};
        float* hi = ops + SBT_B1_FLOATS + (int64_t)(2 * q) * 8192;
        float* lo = hi + 8192;
        sbt_put4(hi, lo, sbt_swz(2 * i, kq), y[0].x, -y[0].y, y[1].x, -y[1].y);
        sbt_put4(hi, lo, sbt_swz(2 * i + 1, kq), y[0].y, y[0].x, y[1].y, y[1].x);
    }
}

// ------------------------------------------------------------------ back-transform
// Warps: eight builders (the A operands and the epilogue), one producer (the B operands by bulk
// copies) and one MMA warp.  Shared memory: a ring of two A slots (a chunk's two A pieces,
// 2 x 16 KB) and a ring of four B slots of 32 KB; a product-(1) chunk's B takes one slot (its two
// 16 KB pieces), a product-(2) chunk's B two (one 32 KB piece each).  mbarriers: A slot full
// (one arrival per builder warp, after each thread's proxy fence) and free (the MMA warp's
// commit), B slot full (the copies' byte count) and free (commit), and one per product done
// (commit).  The builders proceed in order (block by block: product (1)'s A, product (2)'s A
// from TMEM, the epilogue), so an A-full arrival also tells the MMA warp that their earlier TMEM
// reads are complete: product (1) accumulates in columns 256..511 and product (2) in 0..255, and
// a block's products overwrite them only after the builders have moved past the reads.  The
// builders meet at one named barrier per block (the next window shares rows with this one).
#define SBT_ASLOT 32768u
#define SBT_BSLOT 32768u
#define SBT_BSLOTS 4
#define SBT_CTA (SBT_THREADS + 64)  // builders + producer warp + MMA warp
// barrier indices
#define SB_AFULL 0   // [2]
#define SB_AFREE 2   // [2]
#define SB_BFULL 4   // [4]
#define SB_BFREE 8   // [4]
#define SB_ACC1 12
#define SB_ACC2 13
#define SB_NBAR 14

__device__ __forceinline__ void sbt_ld16(uint32_t ta, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(ta));
}
__device__ __forceinline__ void sbt_bar() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
__device__ __forceinline__ void sbt_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(b))
                 : "memory");
}

// bounded wait that also gives up once the CTA has failed
__device__ __forceinline__ bool sbt_wait(uint64_t* bar, uint32_t parity, volatile int* fail) {
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
        if ((it & 255u) == 255u && *fail) return false;
    }
    *fail = 1;
    return false;
}

// a builder warp has written its part of A slot s: each thread fences its stores for the async
// proxy (and orders its earlier TMEM reads), then one arrival per warp
__device__ __forceinline__ void sbt_arrive_a(uint64_t* bar) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncwarp();
    if ((threadIdx.x & 31) == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// loads of one product-(1) chunk's A values: column c, window rows 16 q + 8 hh .. + 7
__device__ __forceinline__ void sbt_load_z(float2* z, const float2* __restrict__ Z, int n, int R0, int nrows, int c,
                                           int q, int hh) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = 16 * q + 8 * hh + u;
        z[u] = (c < n && i < nrows) ? Z[(int64_t)(R0 + i) * n + c] : make_float2(0.f, 0.f);
    }
}
// old values of one epilogue part: column c, window rows ib .. ib + 15
__device__ __forceinline__ void sbt_load_part(float2* zo, const float2* __restrict__ Z, int n, int R0, int nrows,
                                              int c, int ib) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
        const int i = ib + u;
        zo[u] = (c < n && i < nrows) ? Z[(int64_t)(R0 + i) * n + c] : make_float2(0.f, 0.f);
    }
}

// A operand chunk q (K' entries 32 q .. 32 q + 31) from the sum of product (1)'s two TMEM
// accumulators: warp w holds TMEM lanes (rows) 32 (w % 4) .. +31 and K' half w / 4.
__device__ __forceinline__ void sbt_a_from_tmem(uint32_t tmem, float* ahi, float* alo, int q) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int row = 32 * (warp & 3) + lane, h = warp >> 2;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    uint32_t u[16], v[16];
    sbt_ld16(tmem + lanes + 256u + 32u * q + 16u * h, u);
    sbt_ld16(tmem + lanes + 384u + 32u * q + 16u * h, v);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 4; ++k)
        sbt_put4(ahi, alo, sbt_swz(row, 4 * h + k), __uint_as_float(u[4 * k]) + __uint_as_float(v[4 * k]),
                 __uint_as_float(u[4 * k + 1]) + __uint_as_float(v[4 * k + 1]),
                 __uint_as_float(u[4 * k + 2]) + __uint_as_float(v[4 * k + 2]),
                 __uint_as_float(u[4 * k + 3]) + __uint_as_float(v[4 * k + 3]));
}

// window of pass s, block g
struct SbtWin {
    int R0, nrows;
};
__device__ __forceinline__ SbtWin sbt_win(int n, int b, int s, int g) {
    const int jhi = n - 2 - s * b - SBT_NB * g, jlo = max(0, jhi - (SBT_NB - 1));
    SbtWin w;
    w.R0 = jlo + 1 + s * b;
    w.nrows = min(jhi - jlo + b, n - w.R0);  // rows the block changes
    return w;
}

__global__ void __launch_bounds__(SBT_CTA, 1) k_sbr_bt_tc(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                        void* __restrict__ pool, const double* __restrict__ Yg,
                                                        double* __restrict__ work, int* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char sbt_smem[];
    __shared__ uint64_t bar[SB_NBAR];
    __shared__ uint32_t tmem_s;
    __shared__ int fail_s;
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n, b = d.band;
    const int c0 = blockIdx.x * 128;
    if (c0 >= n) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    unsigned char* base = (unsigned char*)(((uintptr_t)sbt_smem + 1023) & ~(uintptr_t)1023);
    unsigned char* As = base;
    unsigned char* Bs = base + 2 * SBT_ASLOT;
    volatile int* fail = &fail_s;
    if (tid == 0) {
        for (int q = 0; q < 2; ++q) {
            mbar_init(&bar[SB_AFULL + q], SBT_THREADS / 32);  // one arrival per builder warp
            mbar_init(&bar[SB_AFREE + q], 1);
        }
        for (int q = 0; q < SBT_BSLOTS; ++q) {
            mbar_init(&bar[SB_BFULL + q], 1);
            mbar_init(&bar[SB_BFREE + q], 1);
        }
        mbar_init(&bar[SB_ACC1], 1);
        mbar_init(&bar[SB_ACC2], 1);
        fail_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_s)),
                     "r"(SBT_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_s;
    const int np = sbr_passes(n, b);
    const float* ops_all = sbt_ops(pool, d);

    if (warp == SBT_THREADS / 32) {
        // producer: the B pieces of every chunk, in the products' order, as slots free up
        if (lane == 0) {
            bool ok = true;
            uint32_t pos = 0;
            int64_t blk = 0;
            for (int s = 0; s < np && ok; ++s) {
                const int nbs = sbt_nblk(n, b, s);
                for (int g = 0; g < nbs && ok; ++g, ++blk) {
                    const float* ops = ops_all + blk * (int64_t)SBT_OPS_FLOATS;
                    for (int q = 0; q < 12 && ok; ++q) {
                        const int nsl = q < 8 ? 1 : 2;
                        for (int k = 0; k < nsl && ok; ++k, ++pos) {
                            const uint32_t sl = pos % SBT_BSLOTS, use = pos / SBT_BSLOTS;
                            if (use > 0 && !(ok = sbt_wait(&bar[SB_BFREE + sl], (use - 1) & 1u, fail))) break;
                            const uint32_t fb = smem_u32(&bar[SB_BFULL + sl]);
                            const uint32_t dst = smem_u32(Bs + sl * SBT_BSLOT);
                            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(SBT_BSLOT)
                                         : "memory");
                            // (1): the chunk's two 16 KB pieces in one slot; (2): piece k, 32 KB
                            const float* src = q < 8 ? ops + (int64_t)(2 * q) * 4096
                                                     : ops + SBT_B1_FLOATS + (int64_t)(2 * (q - 8) + k) * 8192;
                            const uint32_t part = q < 8 ? 16384u : 32768u;
                            asm volatile(
                                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                    dst),
                                "l"(src), "r"(part), "r"(fb)
                                : "memory");
                            if (q < 8)
                                asm volatile(
                                    "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                                        dst + 16384u),
                                    "l"(src + 4096), "r"(16384u), "r"(fb)
                                    : "memory");
                        }
                    }
                }
            }
        }
    } else if (warp == SBT_THREADS / 32 + 1) {
        // MMA warp: each chunk's 12 products once its A and B pieces are in
        if (lane == 0) {
            bool ok = true;
            uint32_t chunk = 0, pos = 0;
            for (int s = 0; s < np && ok; ++s) {
                const int nbs = sbt_nblk(n, b, s);
                for (int g = 0; g < nbs && ok; ++g) {
                    for (int q = 0; q < 12 && ok; ++q, ++chunk) {
                        const int nb = q < 8 ? 1 : 2;
                        const uint32_t sl = chunk & 1u, s0 = pos % SBT_BSLOTS, s1 = (pos + 1) % SBT_BSLOTS;
                        ok = sbt_wait(&bar[SB_AFULL + sl], (chunk >> 1) & 1u, fail) &&
                             sbt_wait(&bar[SB_BFULL + s0], (pos / SBT_BSLOTS) & 1u, fail) &&
                             (nb == 1 || sbt_wait(&bar[SB_BFULL + s1], ((pos + 1) / SBT_BSLOTS) & 1u, fail));
                        if (!ok) break;
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = smem_u32(As + sl * SBT_ASLOT);
                        const uint32_t sb0 = smem_u32(Bs + s0 * SBT_BSLOT), sb1 = smem_u32(Bs + s1 * SBT_BSLOT);
                        const uint64_t a1 = umma_desc(sa), a2 = umma_desc(sa + 16384u);
                        const uint64_t b1 = umma_desc(sb0), b2 = umma_desc(nb == 2 ? sb1 : sb0 + 16384u);
                        const uint32_t N = q < 8 ? 128u : 256u;
                        const uint32_t idesc = umma_idesc_mn(2, 128u, N);
                        const uint32_t dacc = q < 8 ? tmem + 256u + 128u * (uint32_t)(q >> 2) : tmem;
                        const bool first = q < 8 ? (q & 3) == 0 : q == 8;
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t adv = (uint64_t)((kk * 32) >> 4);
                            const uint64_t pa[3] = {a1, a1, a2}, pb[3] = {b1, b2, b1};
#pragma unroll
                            for (int pp = 0; pp < 3; ++pp) {
                                const uint32_t accf = (!first || kk > 0 || pp > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
                                    "l"(pa[pp] + adv), "l"(pb[pp] + adv), "r"(idesc), "r"(accf)
                                    : "memory");
                            }
                        }
                        sbt_commit(&bar[SB_AFREE + sl]);
                        sbt_commit(&bar[SB_BFREE + s0]);
                        if (nb == 2) sbt_commit(&bar[SB_BFREE + s1]);
                        if (q == 7) sbt_commit(&bar[SB_ACC1]);
                        if (q == 11) sbt_commit(&bar[SB_ACC2]);
                        pos += nb;
                    }
                }
            }
        }
    } else {
        // builders
        const double* Y = Yg + d.sq_off;
        float2* Z = reinterpret_cast<float2*>(sbr_zbase(work, d));
        {  // Z = Y on this slab (every row; row 0 is touched by no reflector)
            const int c = c0 + (tid & 127);
            if (c < n)
                for (int r = tid >> 7; r < n; r += SBT_THREADS / 128)
                    Z[(int64_t)r * n + c] = make_float2((float)Y[(int64_t)r * n + c], 0.f);
        }
        sbt_bar();
        const int r = tid & 127, hh = tid >> 7;  // product (1): A row r = slab column c0 + r, rows half hh
        const int c = c0 + 32 * (warp & 3) + lane, h = warp >> 2;  // epilogue: column, window rows 64 h ..
        uint32_t chunk = 0, pacc = 0;
        float2 z[8];
        bool zpre = false;
        bool stop = false;
        for (int s = 0; s < np && !stop; ++s) {
            const int nbs = sbt_nblk(n, b, s);
            for (int g = 0; g < nbs && !stop; ++g) {
                const SbtWin W = sbt_win(n, b, s, g);
                if (!zpre) sbt_load_z(z, Z, n, W.R0, W.nrows, c0 + r, 0, hh);
                // (1) W^T = Z_R^T conj(V): 8 chunks of 16 window rows
                for (int q = 0; q < 8; ++q, ++chunk) {
                    const uint32_t sl = chunk & 1u, use = chunk >> 1;
                    if (use > 0) (void)sbt_wait(&bar[SB_AFREE + sl], (use - 1) & 1u, fail);
                    float* ahi = reinterpret_cast<float*>(As + sl * SBT_ASLOT);
                    float* alo = ahi + 4096;
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        sbt_put4(ahi, alo, sbt_swz(r, 4 * hh + k), z[2 * k].x, z[2 * k].y, z[2 * k + 1].x,
                                 z[2 * k + 1].y);
                    if (q < 7) sbt_load_z(z, Z, n, W.R0, W.nrows, c0 + r, q + 1, hh);  // in flight meanwhile
                    sbt_arrive_a(&bar[SB_AFULL + sl]);
                }
                (void)sbt_wait(&bar[SB_ACC1], pacc, fail);
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // (2) Z_R^T -= W^T Y^T (N = 256: 128 window rows, Re and Im): 4 chunks of 16 j
                for (int q = 0; q < 4; ++q, ++chunk) {
                    const uint32_t sl = chunk & 1u, use = chunk >> 1;
                    if (use > 0) (void)sbt_wait(&bar[SB_AFREE + sl], (use - 1) & 1u, fail);
                    float* ahi = reinterpret_cast<float*>(As + sl * SBT_ASLOT);
                    sbt_a_from_tmem(tmem, ahi, ahi + 4096, q);
                    sbt_arrive_a(&bar[SB_AFULL + sl]);
                }
                // epilogue: Z_R -= U; the old values of the first part, and (when they do not lie in
                // this window) the next block's first A rows, load while the products finish
                float2 zo[16];
                sbt_load_part(zo, Z, n, W.R0, W.nrows, c, 64 * h);
                const bool more = g + 1 < nbs || s + 1 < np;
                zpre = false;
                if (more) {
                    const SbtWin Wn = g + 1 < nbs ? sbt_win(n, b, s, g + 1) : sbt_win(n, b, s + 1, 0);
                    if (Wn.R0 + 16 <= W.R0 || Wn.R0 >= W.R0 + W.nrows) {
                        sbt_load_z(z, Z, n, Wn.R0, Wn.nrows, c0 + r, 0, hh);
                        zpre = true;
                    }
                }
                (void)sbt_wait(&bar[SB_ACC2], pacc, fail);
                pacc ^= 1u;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll 1
                for (int part = 0; part < 4; ++part) {
                    const int ib = 64 * h + 16 * part;  // window rows ib .. ib + 15
                    uint32_t v[2][16];
                    sbt_ld16(tmem + lanes + (uint32_t)(2 * ib), v[0]);
                    sbt_ld16(tmem + lanes + (uint32_t)(2 * ib + 16), v[1]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    float2 zn[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u)
                        zn[u] = make_float2(zo[u].x - __uint_as_float(v[u >> 3][2 * (u & 7)]),
                                            zo[u].y - __uint_as_float(v[u >> 3][2 * (u & 7) + 1]));
                    if (part < 3) sbt_load_part(zo, Z, n, W.R0, W.nrows, c, ib + 16);
#pragma unroll
                    for (int u = 0; u < 16; ++u) {
                        const int i = ib + u;
                        if (c < n && i < W.nrows) Z[(int64_t)(W.R0 + i) * n + c] = zn[u];
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                sbt_bar();  // the window's rows are written before the next block reads them
                stop = *fail != 0;  // read by every builder after the same barrier
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    // on a failure, give the copies and products in flight a bounded time to land before the
    // shared memory and TMEM are released (each wait ends on its own limit)
    if (fail_s && tid == 0)
        for (int k = 0; k < SB_NBAR; ++k) (void)mbar_wait(&bar[k], 0u), (void)mbar_wait(&bar[k], 1u);
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(SBT_TMEM_COLS) : "memory");
    if (fail_s && tid == 0) status[sid] = MMF_ST_NOCONV;
}

size_t mmf_sbt_smem() { return 1024 + 2 * (size_t)SBT_ASLOT + SBT_BSLOTS * (size_t)SBT_BSLOT; }

cudaError_t mmf_launch_sbr_bt_tc(const MmfLaunch& L, const double2* store, const double* Y, double* work, void* pool,
                                 float2* Zout, int* status) {
    if (L.count <= 0) return cudaSuccess;
    const size_t sm = mmf_sbt_smem();
    cudaError_t e = cudaFuncSetAttribute(k_sbr_wy, cudaFuncAttributeMaxDynamicSharedMemorySize, SBT_WY_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_sbr_bt_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    // most blocks any system of the launch has: n = nmax at the narrowest band of the class (33)
    const int nb_max = (int)sbt_blocks(L.nmax, 33);
    k_sbr_wy<<<dim3(nb_max, L.count), 256, SBT_WY_SMEM, L.stream>>>(L.desc, L.idx, store, pool);
    k_sbr_bt_tc<<<dim3((L.nmax + 127) / 128, L.count), SBT_CTA, sm, L.stream>>>(L.desc, L.idx, pool, Y, work, status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return mmf_launch_sbr_out(L, work, Zout);
}
