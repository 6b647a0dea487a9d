// k_hetrd.cu -- S2: blocked complex Householder reduction of H_F to real tridiagonal form.
//
// The paper hands this step to LAPACK (Sec. 3.2); this is our own GPU formulation of the
// standard blocked reduction (Dongarra, Sorensen & Hammarling 1989).  Lower storage,
// column-major; only the lower triangle is read or updated.
//
// For column k the reflector P_k = I - tau_k v v^H (v[k+1] = 1, v[r] = 0 for r <= k)
// satisfies P_k^H A(k+1:, k) = beta_k e_1 with beta_k real:
//     beta = -sign(Re alpha) sqrt(|alpha|^2 + ||x||^2),  tau = (beta - alpha) / beta,
//     v[k+2:] = x / (alpha - beta)        (alpha = A(k+1, k), x = A(k+2:, k)).
// Two-sided update A <- P^H A P = A - v w^H - w v^H with
//     y = A v,   w = tau y - (1/2) |tau|^2 (v^H y) v.
// Within a panel of NB columns the updates are deferred (V, W kept in global workspace):
// before its reflector, column k receives A(k:, k) -= V W(k,:)^H + W V(k,:)^H, and
// y = A22 v - V (W^H v) - W (V^H v).  After the panel the trailing lower triangle
// receives A -= V W^H + W V^H (her2k).
// Result: d (diagonal), e = beta (sub-diagonal, real), tau, and v[k+2:] stored in
// A(k+2:, k).  Q = P_0 P_1 ... P_{n-2}, Q^H H_F Q = tridiag(e, d, e).
//
// One thread-block cluster of CL CTAs (512 threads each) per system.  The hemv streams the
// lower triangle of the trailing matrix once per column with coalesced column reads: a warp
// owns 8 columns, lanes own rows, the row part accumulates through shared-memory atomics and
// the column part by warp-shuffle reductions.  With CL = 2 the two CTAs of the cluster split the
// column blocks of the hemv, the rows of the column update and the tiles of the trailing
// update; each adds its partner's partial hemv result through distributed shared memory and
// repeats the short O(m) vector steps itself.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mmf_internal.h"
#include "umma_common.h"

namespace cg = cooperative_groups;

#define HT_THREADS 512
#define HT_TILE 64
#define HT_SEG 512   // rows per hemv task (a multiple of 64)

template <class R>
__device__ __forceinline__ R block_sum(R v, R* red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        R s = (threadIdx.x < HT_THREADS / 32) ? red[threadIdx.x] : R(0);
        s = warp_sum(s);
        if (threadIdx.x == 0) red[32] = s;
    }
    __syncthreads();
    R r = red[32];
    __syncthreads();
    return r;
}


// FP32 hemv pipeline: per warp two stages of HT_CH rows x 8 columns, filled by cp.async
#define HT_CH 64
#define HT_STAGE_ELEMS (8 * HT_CH)

template <class R>
__host__ __device__ constexpr size_t ht_fixed_bytes() {
    return sizeof(typename Cx<R>::T) * (4 * MMF_NB + 4) + sizeof(R) * 72;
}
template <class R>
__host__ __device__ inline size_t ht_big_offset(int nmax) {
    const size_t o = sizeof(typename Cx<R>::T) * 3 * (size_t)nmax + ht_fixed_bytes<R>();
    return (o + 15) & ~(size_t)15;
}
// FP32: the hemv's cp.async stages, or (tensor-core trailing update) two operand stages of 64 KB
// at a 1024-byte boundary
#define HT_TC_STAGE 65536u
template <class R>
__host__ __device__ constexpr size_t ht_big_bytes() {
    return sizeof(R) == 4 ? (size_t)(HT_THREADS / 32) * 2 * HT_STAGE_ELEMS * sizeof(typename Cx<R>::T) + 1024
                          : (size_t)4 * MMF_NB * HT_TILE * sizeof(typename Cx<R>::T);
}
static_assert((HT_THREADS / 32) * 2 * HT_STAGE_ELEMS * 8 >= 2 * HT_TC_STAGE, "tensor-core stages fit");

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc, int src_bytes) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gsrc), "r"(src_bytes) : "memory");
}
static_assert(4 * MMF_NB * HT_TILE <= (HT_THREADS / 32) * 2 * HT_STAGE_ELEMS, "her2k tiles fit the hemv stages");

// two block-wide sums in one pass (red holds 2 x 33 values)
template <class R>
__device__ __forceinline__ void block_sum2(R a, R b, R* red, R& sa, R& sb) {
    a = warp_sum(a);
    b = warp_sum(b);
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = a;
        red[33 + (threadIdx.x >> 5)] = b;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        R x = (threadIdx.x < HT_THREADS / 32) ? red[threadIdx.x] : R(0);
        R y = (threadIdx.x < HT_THREADS / 32) ? red[33 + threadIdx.x] : R(0);
        x = warp_sum(x);
        y = warp_sum(y);
        if (threadIdx.x == 0) {
            red[32] = x;
            red[65] = y;
        }
    }
    __syncthreads();
    sa = red[32];
    sb = red[65];
    __syncthreads();
}

__device__ __forceinline__ void atomic_add_c(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_add_c(float2* p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}


// FP32 hemv share of one warp, pipelined through shared memory: the warp's chunks (HT_CH rows x
// 8 columns of its row-segment tasks) are copied by cp.async one chunk ahead of the arithmetic,
// so the trailing matrix streams while the previous chunk is multiplied.  Task h of the CTA:
// column block (rank + CL (h % nloc)) of 8 columns, rows from segment h / nloc (HT_SEG rows).
// The arithmetic is branch-free outside the diagonal chunk: the block's 8 entries of v are held
// in registers per task, the chunk's operands are read from shared memory before the FMAs.
// Complex products use packed FP32 pair FMAs with split accumulators: for a row r,
// y_r += sum_jj a v_jj is kept as r1 = sum a (v.x, v.x), r2 = sum a (v.y, v.y), y_r += (r1.x - r2.y,
// r1.y + r2.x); for a column, sum_r conj(a) v_r as c1 = sum a (v_r.x, v_r.x), c2 = sum a (v_r.y,
// v_r.y), added as (c1.x + c2.y, c2.x - c1.y).
struct HtTask {
    int c0, rbeg, rend, nc;
};

__device__ __forceinline__ bool ht_task(int h, int nloc, int rank, int CL, int m, HtTask& t) {
    const int qb = h % nloc, sg = h / nloc;
    t.c0 = (rank + CL * qb) << 3;
    t.rbeg = t.c0 + sg * HT_SEG;
    t.rend = min(t.rbeg + HT_SEG, m);
    t.nc = min(8, m - t.c0);
    return t.rbeg < m;
}

__device__ __forceinline__ void ht_issue(const float2* __restrict__ a22, int ld, const HtTask& t, int r0,
                                         float2* buf, int lane) {
    const float2* colbase = a22 + (int64_t)t.c0 * ld;
    if (r0 >= t.c0 + 8 && r0 + HT_CH <= t.rend && t.nc == 8) {
        // the common chunk: below the diagonal block, inside the task, all 8 columns present
        const float2* p = colbase + r0 + lane;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj)
#pragma unroll
            for (int hf = 0; hf < HT_CH / 32; ++hf)
                cp_async8(buf + jj * HT_CH + lane + 32 * hf, p + (int64_t)jj * ld + 32 * hf, 8);
        asm volatile("cp.async.commit_group;" ::: "memory");
        return;
    }
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
#pragma unroll
        for (int hf = 0; hf < HT_CH / 32; ++hf) {
            const int row = r0 + lane + 32 * hf;
            const bool ok = jj < t.nc && row < t.rend && row >= t.c0 + jj;
            const float2* src = ok ? colbase + (int64_t)jj * ld + row : a22;
            cp_async8(buf + jj * HT_CH + lane + 32 * hf, src, ok ? 8 : 0);
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ int hemv_f32_staged(const float2* __restrict__ a22, int ld, int m, const float2* __restrict__ vS,
                               float2* yS, float2* stg, int rank, int CL, int nloc, int nseg, int warp, int lane) {
    const int NW = HT_THREADS / 32;
    const int nh = nloc * nseg;
    // the warp's first valid task
    int h = warp;
    HtTask t;
    while (h < nh && !ht_task(h, nloc, rank, CL, m, t)) h += NW;
    if (h >= nh) return 0;
    int r0 = t.rbeg, buf = 0, nchunks = 0;
    ht_issue(a22, ld, t, r0, stg, lane);
    float2 v[8], vxx[8], vyy[8], c1[8], c2[8];
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
        v[jj] = (jj < t.nc) ? vS[t.c0 + jj] : czero<float2>();
        vxx[jj] = make_float2(v[jj].x, v[jj].x);
        vyy[jj] = make_float2(v[jj].y, v[jj].y);
        c1[jj] = c2[jj] = czero<float2>();
    }
    for (;;) {
        ++nchunks;
        // next chunk: the rest of this task, else the next valid task
        int hn = h, r0n = r0 + HT_CH;
        HtTask tn = t;
        if (r0n >= t.rend) {
            hn = h + NW;
            while (hn < nh && !ht_task(hn, nloc, rank, CL, m, tn)) hn += NW;
            r0n = tn.rbeg;
        }
        const bool more = hn < nh;
        if (more) {
            ht_issue(a22, ld, tn, r0n, stg + (buf ^ 1) * HT_STAGE_ELEMS, lane);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncwarp();
        const float2* sb = stg + buf * HT_STAGE_ELEMS;
        const bool diag = r0 < t.c0 + 8;  // the chunk holds the diagonal entries of the block
#pragma unroll
        for (int hf = 0; hf < HT_CH / 32; ++hf) {
            const int r = r0 + lane + 32 * hf;
            float2 a[8];
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) a[jj] = sb[jj * HT_CH + lane + 32 * hf];  // 0 where not loaded
            const float2 vr = (r < t.rend) ? vS[r] : czero<float2>();
            float2 ra = czero<float2>();
            const float2 vrx = make_float2(vr.x, vr.x), vry = make_float2(vr.y, vr.y);
            if (!diag) {
                float2 r1 = make_float2(0.f, 0.f), r2 = r1;
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    r1 = __ffma2_rn(a[jj], vxx[jj], r1);
                    r2 = __ffma2_rn(a[jj], vyy[jj], r2);
                    c1[jj] = __ffma2_rn(a[jj], vrx, c1[jj]);
                    c2[jj] = __ffma2_rn(a[jj], vry, c2[jj]);
                }
                ra = make_float2(r1.x - r2.y, r1.y + r2.x);
            } else {
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    const int c = t.c0 + jj;
                    if (r > c) {
                        ra = ra + a[jj] * v[jj];
                        c1[jj] = __ffma2_rn(a[jj], vrx, c1[jj]);
                        c2[jj] = __ffma2_rn(a[jj], vry, c2[jj]);
                    } else if (r == c) {
                        ra = ra + a[jj].x * v[jj];
                    }
                }
            }
            if (r < t.rend) atomic_add_c(&yS[r], ra);
        }
        __syncwarp();  // every lane is done with this stage before it is refilled
        if (hn != h || !more) {  // the task is complete: add its column part
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                // conj(a) vr summed: (c1.x + c2.y, c2.x - c1.y)
                const float sx = warp_sum(c1[jj].x + c2[jj].y), sy = warp_sum(c2[jj].x - c1[jj].y);
                if (lane == 0 && jj < t.nc) atomic_add_c(&yS[t.c0 + jj], mk(sx, sy));
                c1[jj] = c2[jj] = czero<float2>();
            }
            if (!more) break;
#pragma unroll
            for (int jj = 0; jj < 8; ++jj) {
                v[jj] = (jj < tn.nc) ? vS[tn.c0 + jj] : czero<float2>();
                vxx[jj] = make_float2(v[jj].x, v[jj].x);
                vyy[jj] = make_float2(v[jj].y, v[jj].y);
            }
        }
        h = hn;
        t = tn;
        r0 = r0n;
        buf ^= 1;
    }
    return nchunks;
}

// ------------------------------------------------------------------ trailing update, tensor cores
// A(c0:, c0:) -= V W^H + W V^H on the lower triangle (FP32 path), as real split-TF32 products on
// the tcgen05 engine.  Tiles of 128 rows x 64 complex columns: column block cb = c0 + 64 tj, row
// blocks rb = cb + 128 ti (the first holds the block's diagonal; entries above it are dropped).
// With K' = 128 real entries per row in four chunks of 32 (the panel's columns), ordered
// (Re V, Im V, Re W, Im W),
//     A'(r)       = [Re V(r,:), Im V(r,:), Re W(r,:), Im W(r,:)]
//     B'(2j)      = [Re W(c,:), Im W(c,:), Re V(c,:), Im V(c,:)]        (c = cb + j)
//     B'(2j + 1)  = [-Im W(c,:), Re W(c,:), -Im V(c,:), Re V(c,:)]
// the product D = A' B'^T holds Re and Im of (V W^H + W V^H)(r, c) in columns 2j and 2j + 1
// (Re(a conj b) = ar br + ai bi, Im(a conj b) = ai br - ar bi).  Each operand is split into TF32
// pieces x = x1 + x2 and each chunk's D = A1 B1^T + A1 B2^T + A2 B1^T goes to its own TMEM
// accumulator (4 x 128 columns), which the epilogue sums in FP32 registers: the tensor cores'
// accumulation is cut to 96 terms, and the result stays within a few FP32 roundings of the
// FP32 units' update.  Chunks 0-1 (the V pass) and 2-3 (the W pass) take the same complex
// values: a thread loads its pass's values once (L2) and builds both chunks from registers into
// one of two 64 KB stages, in the tensor cores' layout (K-major, 128-byte swizzle); one thread
// issues each chunk's 12 tcgen05.mma (M = 128, N = 128, K = 8) and commits them to the stage's
// mbarrier, so that the next chunk is built while they run.  Epilogue: warp w reads TMEM lanes
// 32 (w % 4) .. +31 (rows) and columns 32 (w / 4) .. +31 (16 complex columns) of each
// accumulator and subtracts the sum from A, whose old values it loaded when the tile began.
// Every wait is bounded; a wait that gives up makes the routine return false.
#define HT_TC_COLS 512u   // TMEM columns: four 128-column accumulators
struct HtTc {
    unsigned char* st;   // two stages of HT_TC_STAGE bytes (1024-byte aligned)
    uint64_t* bar;       // [0], [1]: stage free; [2]: tile's products done
    uint32_t tmem;
    uint32_t used[2], waited[2], pacc;
};

__device__ __forceinline__ void ht_split4(float* hi, float* lo, int off, float x0, float x1, float x2, float x3) {
    const float4 h = make_float4(tf32_round(x0), tf32_round(x1), tf32_round(x2), tf32_round(x3));
    *reinterpret_cast<float4*>(hi + off) = h;
    *reinterpret_cast<float4*>(lo + off) =
        make_float4(tf32_round(x0 - h.x), tf32_round(x1 - h.y), tf32_round(x2 - h.z), tf32_round(x3 - h.w));
}

__device__ __forceinline__ void ht_tmem_ld32(uint32_t ta, uint32_t* v) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(ta));
}

// Tiles are dealt round-robin over nshare CTAs (this one takes those with index % nshare ==
// share); full = true would update both triangles (full Hermitian storage: row blocks from c0,
// no triangle mask).
__device__ bool her2k_tc(float2* __restrict__ A, int ld, int n, int c0, const float2* __restrict__ V,
                         const float2* __restrict__ W, int nb, int nshare, int share, bool full, HtTc& T) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t idesc = umma_idesc_mn(2, 128u, 128u);  // TF32 x TF32 -> F32, M = N = 128
    const int ncb = (n - c0 + 63) / 64;
    int tcount = 0;
    bool ok = true;
    for (int tj = 0; tj < ncb && ok; ++tj) {
        const int cb = c0 + 64 * tj;
        for (int rb = full ? c0 : cb; rb < n && ok; rb += 128) {
            if ((tcount++ % nshare) != share) continue;
            // old values of this thread's 16 entries (row r, columns cc .. cc + 15), in flight
            // while the operands are built
            const int r = rb + 32 * (warp & 3) + lane, cc = cb + 16 * (warp >> 2);
            float2 old[16];
#pragma unroll
            for (int q = 0; q < 16; ++q)
                old[q] = (r < n && cc + q < n && (full || r >= cc + q)) ? A[r + (int64_t)(cc + q) * ld]
                                                                         : make_float2(0.f, 0.f);
            for (int pass = 0; pass < 2 && ok; ++pass) {
                const float2* P = pass ? W : V;   // A' source
                const float2* Q = pass ? V : W;   // B' source
                // items e = tid, tid + 512: operand row rr = e % 128 (lanes over rows: coalesced
                // column reads), K group kq = e / 128 (4 panel columns)
                float2 a[2][4], b[2][4];
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const int e = tid + it * HT_THREADS, rr = e & 127, kq = e >> 7;
                    const int ra = rb + rr, cbr = cb + (rr >> 1);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int p = 4 * kq + u;
                        a[it][u] = (p < nb && ra < n) ? P[ra + (int64_t)p * ld] : make_float2(0.f, 0.f);
                        b[it][u] = (p < nb && cbr < n) ? Q[cbr + (int64_t)p * ld] : make_float2(0.f, 0.f);
                    }
                }
                for (int half = 0; half < 2 && ok; ++half) {
                    const int kc = 2 * pass + half, s = half;
                    if (T.used[s] > T.waited[s]) {  // the products that last read this stage are done
                        ok = __syncthreads_and(mbar_wait(&T.bar[s], T.waited[s] & 1u) ? 1 : 0) != 0;
                        ++T.waited[s];
                        if (!ok) break;
                    }
                    float* ahi = reinterpret_cast<float*>(T.st + s * HT_TC_STAGE);
                    float* alo = ahi + 4096;
                    float* bhi = alo + 4096;
                    float* blo = bhi + 4096;
#pragma unroll
                    for (int it = 0; it < 2; ++it) {
                        const int e = tid + it * HT_THREADS, rr = e & 127, kq = e >> 7;
                        const int off = (rr >> 3) * 256 + (rr & 7) * 32 + ((kq ^ (rr & 7)) << 2);
                        // A': Re (half 0) or Im (half 1) of the pass's matrix; B' row rr (column
                        // cb + rr / 2): Re row (rr even) [Re, Im] of the other matrix over the two
                        // halves, Im row (rr odd) [-Im, Re]
                        const int h = rr & 1;
                        float x[4], y[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            x[u] = half ? a[it][u].y : a[it][u].x;
                            y[u] = h ? (half ? b[it][u].x : -b[it][u].y) : (half ? b[it][u].y : b[it][u].x);
                        }
                        ht_split4(ahi, alo, off, x[0], x[1], x[2], x[3]);
                        ht_split4(bhi, blo, off, y[0], y[1], y[2], y[3]);
                    }
                    // the stores above are read by the tensor cores' async proxy
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncthreads();
                    if (tid == 0) {
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t sa = smem_u32(ahi);
                        const uint64_t a1 = umma_desc(sa), a2 = umma_desc(sa + 16384u);
                        const uint64_t b1 = umma_desc(sa + 32768u), b2 = umma_desc(sa + 49152u);
                        const uint32_t dacc = T.tmem + 128u * (uint32_t)kc;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {  // 32 bytes (8 TF32) of K per instruction
                            const uint64_t adv = (uint64_t)((q * 32) >> 4);
                            const uint64_t pa[3] = {a1, a1, a2}, pb[3] = {b1, b2, b1};
#pragma unroll
                            for (int pp = 0; pp < 3; ++pp) {
                                const uint32_t accf = (q > 0 || pp > 0) ? 1u : 0u;
                                asm volatile(
                                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                    "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dacc),
                                    "l"(pa[pp] + adv), "l"(pb[pp] + adv), "r"(idesc), "r"(accf)
                                    : "memory");
                            }
                        }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                         smem_u32(&T.bar[s]))
                                     : "memory");
                        if (kc == 3)
                            asm volatile(
                                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                    smem_u32(&T.bar[2]))
                                : "memory");
                    }
                    ++T.used[s];
                }
            }
            if (!ok) break;
            ok = __syncthreads_and(mbar_wait(&T.bar[2], T.pacc) ? 1 : 0) != 0;
            T.pacc ^= 1u;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t ta = T.tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(32 * (warp >> 2));
            float2 acc[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll
            for (int kc = 0; kc < 4; ++kc) {
                uint32_t v[32];
                ht_tmem_ld32(ta + 128u * (uint32_t)kc, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    acc[q].x += __uint_as_float(v[2 * q]);
                    acc[q].y += __uint_as_float(v[2 * q + 1]);
                }
            }
#pragma unroll
            for (int q = 0; q < 16; ++q)
                if (r < n && cc + q < n && (full || r >= cc + q))
                    A[r + (int64_t)(cc + q) * ld] = make_float2(old[q].x - acc[q].x, old[q].y - acc[q].y);
            // the next tile's first products overwrite the accumulators after the next barrier
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        }
    }
    return ok;
}

template <class R, int CL, bool TC>
__global__ void __launch_bounds__(HT_THREADS, 1)
k_hetrd(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
        typename Cx<R>::T* __restrict__ H, typename Cx<R>::T* __restrict__ Vpool,
        typename Cx<R>::T* __restrict__ Wpool, double* __restrict__ dvec,
        double* __restrict__ evec, typename Cx<R>::T* __restrict__ taupool, int nmax,
        int* __restrict__ status) {
    static_assert(!TC || sizeof(R) == 4, "tensor-core trailing update on the FP32 path only");
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint64_t tc_bar[3];
    __shared__ uint32_t tc_tmem;
    C* vS = reinterpret_cast<C*>(smem_raw);   // nmax
    C* yS = vS + nmax;                          // nmax: this CTA's partial y = A22 v
    C* yF = yS + nmax;                          // nmax: full y (CL = 2)
    C* wk = yF + nmax;                          // MMF_NB
    C* vk = wk + MMF_NB;                        // MMF_NB
    C* xw = vk + MMF_NB;                        // MMF_NB
    C* xv = xw + MMF_NB;                        // MMF_NB
    C* sc = xv + MMF_NB;                        // 4 scalars: tau, scale, alpha2
    R* red = reinterpret_cast<R*>(sc + 4);      // 66 (two block sums at once)
    // one region shared by the her2k staging tiles and (FP32) the hemv's cp.async stages
    C* big = reinterpret_cast<C*>(smem_raw + ht_big_offset<R>(nmax));
    C* tVr = big;                               // MMF_NB x HT_TILE (her2k staging, transposed)
    C* tWr = tVr + MMF_NB * HT_TILE;
    C* tVc = tWr + MMF_NB * HT_TILE;
    C* tWc = tVc + MMF_NB * HT_TILE;

    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (CL > 1) ? (int)cluster.block_rank() : 0;
    const MmfDesc d = descs[idx[blockIdx.x / CL]];
    const int n = d.n, ld = d.ld;
    C* A = H + d.mat_off;
    C* V = Vpool + d.pan_off;
    C* W = Wpool + d.pan_off;
    double* dd = dvec + d.vec_off;
    double* ee = evec + d.vec_off;
    C* tau = taupool + d.vec_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int NW = HT_THREADS / 32;
    HtTc T = {};
    bool tc_ok = true;
    if constexpr (TC) {
        if (tid == 0) {
            for (int q = 0; q < 3; ++q) mbar_init(&tc_bar[q], 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (warp == 0) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tc_tmem)),
                         "r"(HT_TC_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        T.st = reinterpret_cast<unsigned char*>(((uintptr_t)big + 1023) & ~(uintptr_t)1023);
        T.bar = tc_bar;
        T.tmem = tc_tmem;
    }

    for (int j0 = 0; j0 < n; j0 += MMF_NB) {
        const int nb = min(MMF_NB, n - j0);
        for (int i = 0; i < nb; ++i) {
            const int k = j0 + i;
            // (a) pending panel updates of column k
            if (i > 0) {
                if (tid < i) {
                    wk[tid] = conj(W[k + (int64_t)tid * ld]);
                    vk[tid] = conj(V[k + (int64_t)tid * ld]);
                }
                __syncthreads();
                for (int r = k + rank * HT_THREADS + tid; r < n; r += CL * HT_THREADS) {
                    // unrolled so that the panel's loads (L2 latency each) are in flight together
                    C acc = czero<C>(), acc2 = czero<C>();
#pragma unroll 8
                    for (int c = 0; c < i; ++c) {
                        acc = acc + V[r + (int64_t)c * ld] * wk[c];
                        acc2 = acc2 + W[r + (int64_t)c * ld] * vk[c];
                    }
                    A[r + (int64_t)k * ld] = A[r + (int64_t)k * ld] - (acc + acc2);
                }
                if (CL > 1) cluster.sync(); else __syncthreads();
            }
            if (tid == 0 && rank == 0) dd[k] = (double)A[k + (int64_t)k * ld].x;
            if (k == n - 1) break;
            const int m = n - k - 1;
            C* col = A + (int64_t)k * ld;

            // (b) reflector
            R part = 0;
            for (int r = k + 2 + tid; r < n; r += HT_THREADS) part += abs2(col[r]);
            const R xn2 = block_sum(part, red);
            if (tid == 0) {
                C alpha = col[k + 1];
                C t, s;
                R beta;
                if (xn2 == R(0) && alpha.y == R(0)) {
                    t = czero<C>();
                    s = czero<C>();
                    beta = alpha.x;
                } else {
                    beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
                    t = mk((beta - alpha.x) / beta, -alpha.y / beta);
                    C den = mk(alpha.x - beta, alpha.y);  // 1 / (alpha - beta)
                    R dn = abs2(den);
                    s = mk(den.x / dn, -den.y / dn);
                }
                if (rank == 0) {
                    ee[k] = (double)beta;
                    tau[k] = t;
                }
                sc[0] = t;
                sc[1] = s;
            }
            __syncthreads();
            const C tk = sc[0], scale = sc[1];
            for (int r = tid; r < n; r += HT_THREADS) {
                C v;
                if (r <= k) {
                    v = czero<C>();
                } else if (r == k + 1) {
                    v = mk(R(1), R(0));
                } else {
                    v = col[r] * scale;
                    if (CL == 1) col[r] = v;  // with a partner CTA still reading col, stored below
                }
                if (r > k) {
                    vS[r - k - 1] = v;
                    yS[r - k - 1] = czero<C>();
                }
                if (rank == 0) V[r + (int64_t)i * ld] = v;
            }
            __syncthreads();

            // (c) y = A22 v (lower triangle) and (d) x_w = W^H v, x_v = V^H v
            const C* a22 = A + (k + 1) + (int64_t)(k + 1) * ld;
            // Tasks: the 2i dot products (every CTA needs them all), then this CTA's share of the
            // hemv: column blocks of 8 (blocks rank, rank + CL, ...) cut into row segments of
            // HT_SEG rows, so that tasks cost about the same and every warp gets some.
            const int nblk = (m + 7) >> 3;
            const int nloc = (nblk - rank + CL - 1) / CL;
            const int nseg = (m + HT_SEG - 1) / HT_SEG;
            const int ntask = 2 * i + nloc * nseg;
            if constexpr (sizeof(R) == 4) {
                for (int task = warp; task < 2 * i; task += NW) {
                    const int c = task >> 1;
                    const C* P = (task & 1) ? V : W;
                    // unrolled: the loads of the V / W column are independent (L2 latency each)
                    C acc = czero<C>(), acc2 = czero<C>();
#pragma unroll 4
                    for (int rp = lane; rp < m; rp += 64) {
                        acc = acc + cmulc(P[(k + 1 + rp) + (int64_t)c * ld], vS[rp]);
                        if (rp + 32 < m) acc2 = acc2 + cmulc(P[(k + 1 + rp + 32) + (int64_t)c * ld], vS[rp + 32]);
                    }
                    acc = acc + acc2;
                    acc.x = warp_sum(acc.x);
                    acc.y = warp_sum(acc.y);
                    if (lane == 0) ((task & 1) ? xv : xw)[c] = acc;
                }
                (void)hemv_f32_staged(reinterpret_cast<const float2*>(a22), ld, m, reinterpret_cast<const float2*>(vS),
                                reinterpret_cast<float2*>(yS),
                                reinterpret_cast<float2*>(big) + (size_t)warp * 2 * HT_STAGE_ELEMS, rank, CL,
                                nloc, nseg, warp, lane);
            } else
            for (int task = warp; task < ntask; task += NW) {
                if (task < 2 * i) {
                    const int c = task >> 1;
                    const C* P = (task & 1) ? V : W;
                    // unrolled: the loads of the V / W column are independent (L2 latency each)
                    C acc = czero<C>(), acc2 = czero<C>();
#pragma unroll 4
                    for (int rp = lane; rp < m; rp += 64) {
                        acc = acc + cmulc(P[(k + 1 + rp) + (int64_t)c * ld], vS[rp]);
                        if (rp + 32 < m) acc2 = acc2 + cmulc(P[(k + 1 + rp + 32) + (int64_t)c * ld], vS[rp + 32]);
                    }
                    acc = acc + acc2;
                    acc.x = warp_sum(acc.x);
                    acc.y = warp_sum(acc.y);
                    if (lane == 0) ((task & 1) ? xv : xw)[c] = acc;
                    continue;
                }
                const int t = task - 2 * i;
                const int q = t % nloc, sg = t / nloc;
                const int c0 = (rank + CL * q) << 3;
                const int rbeg = c0 + sg * HT_SEG;
                if (rbeg >= m) continue;  // the segment lies below the matrix
                const int rend = min(rbeg + HT_SEG, m);
                const int nc = min(8, m - c0);
                // v of the block's columns is read from shared memory at each use (registers go
                // to the loads in flight)
                C ca[8];
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) ca[jj] = czero<C>();
                int r0 = rbeg;
                if (sg == 0) {  // diagonal chunk (rows c0 .. c0+31)
                    const int r = c0 + lane;
                    if (r < m) {
                        const C vr = vS[r];
                        C ra = czero<C>();
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const int c = c0 + jj;
                            if (jj < nc) {
                                if (r > c) {
                                    C a = a22[r + (int64_t)c * ld];
                                    ra = ra + a * vS[c];
                                    ca[jj] = ca[jj] + cmulc(a, vr);
                                } else if (r == c) {
                                    ra = ra + a22[r + (int64_t)c * ld].x * vS[c];
                                }
                            }
                        }
                        atomic_add_c(&yS[r], ra);
                    }
                    r0 = c0 + 32;
                }
                // strictly-lower chunks of 32 rows (this loop serves the FP64 path, which is bound by
                // the FP64 units; the FP32 path streams through hemv_f32_staged)
                for (; r0 < rend; r0 += 32) {
                    const int rr = r0 + lane;
                    if (rr < rend) {
                        C a[8];
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj)
                            a[jj] = (jj < nc) ? a22[rr + (int64_t)(c0 + jj) * ld] : czero<C>();
                        const C vr = vS[rr];
                        C sa = czero<C>();
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) {
                            const C v = (jj < nc) ? vS[c0 + jj] : czero<C>();
                            sa = sa + a[jj] * v;
                            ca[jj] = ca[jj] + cmulc(a[jj], vr);
                        }
                        atomic_add_c(&yS[rr], sa);
                    }
                }
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) {
                    R sx = warp_sum(ca[jj].x), sy = warp_sum(ca[jj].y);
                    if (lane == 0 && jj < nc) atomic_add_c(&yS[c0 + jj], mk(sx, sy));
                }
            }
            if (CL > 1) {
                cluster.sync();  // both partial y complete
                const C* yP = cluster.map_shared_rank(yS, rank ^ 1);
                for (int rp = tid; rp < m; rp += HT_THREADS) yF[rp] = yS[rp] + yP[rp];
                __syncthreads();
            } else {
                __syncthreads();  // y complete
            }
            const C* yT = (CL > 1) ? yF : yS;

            // (d) corrections, (e) w = tau y - (1/2) tau (w^H v) v
            C dpart = czero<C>();
            for (int rp = tid; rp < m; rp += HT_THREADS) {
                C y = yT[rp], y2 = czero<C>();
#pragma unroll 8
                for (int c = 0; c < i; ++c) {
                    y = y - V[(k + 1 + rp) + (int64_t)c * ld] * xw[c];
                    y2 = y2 + W[(k + 1 + rp) + (int64_t)c * ld] * xv[c];
                }
                y = y - y2;
                C w = tk * y;
                yF[rp] = w;
                dpart = dpart + cmulc(w, vS[rp]);
            }
            R dx, dy;
            block_sum2(dpart.x, dpart.y, red, dx, dy);
            const C alpha2 = R(-0.5) * (tk * mk(dx, dy));
            if (rank == 0)
                for (int r = tid; r < n; r += HT_THREADS) {
                    C w = czero<C>();
                    if (r > k) w = yF[r - k - 1] + alpha2 * vS[r - k - 1];
                    W[r + (int64_t)i * ld] = w;
                }
            if (CL > 1) {
                cluster.sync();  // both CTAs are done with column k
                if (rank == 0)
                    for (int r = k + 2 + tid; r < n; r += HT_THREADS) col[r] = vS[r - k - 1];
            } else {
                __syncthreads();
            }
        }

        // trailing her2k on the lower triangle of A(c0:, c0:)
        const int c0 = j0 + nb;
        if constexpr (TC) {
            if (c0 < n) {
                if (tc_ok)
                    tc_ok = her2k_tc(reinterpret_cast<float2*>(A), ld, n, c0, reinterpret_cast<const float2*>(V),
                                     reinterpret_cast<const float2*>(W), nb, CL, rank, false, T);
                if (CL > 1) cluster.sync();
            }
        } else if (c0 < n) {
            const int nt = (n - c0 + HT_TILE - 1) / HT_TILE;
            const int rr = tid & (HT_TILE - 1), cg = tid / HT_TILE;  // 8 column groups
            int tcount = 0;
            for (int ti = 0; ti < nt; ++ti) {
                for (int tj = 0; tj <= ti; ++tj) {
                    if ((tcount++ % CL) != rank) continue;
                    const int rbase = c0 + ti * HT_TILE, cbase = c0 + tj * HT_TILE;
                    for (int e = tid; e < nb * HT_TILE; e += HT_THREADS) {
                        const int p = e / HT_TILE, q = e - p * HT_TILE;
                        const int r = rbase + q, c = cbase + q;
                        tVr[e] = (r < n) ? V[r + (int64_t)p * ld] : czero<C>();
                        tWr[e] = (r < n) ? W[r + (int64_t)p * ld] : czero<C>();
                        tVc[e] = (c < n) ? conj(V[c + (int64_t)p * ld]) : czero<C>();
                        tWc[e] = (c < n) ? conj(W[c + (int64_t)p * ld]) : czero<C>();
                    }
                    __syncthreads();
                    C acc[8];
                    if constexpr (sizeof(R) == 4) {
                        // packed FP32 pairs: s1 += (a.x, a.x) c + (b.x, b.x) d, s2 += (a.y, a.y) c + (b.y, b.y) d,
                        // so that a c + b d = (s1.x - s2.y, s1.y + s2.x)
                        float2 s1[8], s2[8];
#pragma unroll
                        for (int q = 0; q < 8; ++q) s1[q] = s2[q] = make_float2(0.f, 0.f);
                        for (int p = 0; p < nb; ++p) {
                            const float2 a = tVr[p * HT_TILE + rr], b = tWr[p * HT_TILE + rr];
                            const float2 ax = make_float2(a.x, a.x), ay = make_float2(a.y, a.y);
                            const float2 bx = make_float2(b.x, b.x), by = make_float2(b.y, b.y);
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const int cc = cg + 8 * q;
                                const float2 c = tWc[p * HT_TILE + cc], dv = tVc[p * HT_TILE + cc];
                                s1[q] = __ffma2_rn(ax, c, s1[q]);
                                s1[q] = __ffma2_rn(bx, dv, s1[q]);
                                s2[q] = __ffma2_rn(ay, c, s2[q]);
                                s2[q] = __ffma2_rn(by, dv, s2[q]);
                            }
                        }
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc[q] = mk(s1[q].x - s2[q].y, s1[q].y + s2[q].x);
                    } else {
#pragma unroll
                        for (int q = 0; q < 8; ++q) acc[q] = czero<C>();
                        for (int p = 0; p < nb; ++p) {
                            const C a = tVr[p * HT_TILE + rr], b = tWr[p * HT_TILE + rr];
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const int cc = cg + 8 * q;
                                acc[q] = acc[q] + a * tWc[p * HT_TILE + cc] + b * tVc[p * HT_TILE + cc];
                            }
                        }
                    }
                    const int r = rbase + rr;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const int c = cbase + cg + 8 * q;
                        if (r < n && c < n && r >= c) {
                            C* pa = A + r + (int64_t)c * ld;
                            *pa = *pa - acc[q];
                        }
                    }
                    __syncthreads();
                }
            }
            if (CL > 1) cluster.sync();
        }
    }
    if constexpr (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (warp == 0)
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(T.tmem), "r"(HT_TC_COLS) : "memory");
        // a wait of the tensor-core update that gave up (the system's reduction is then incomplete)
        if (!tc_ok && tid == 0) status[idx[blockIdx.x / CL]] = MMF_ST_NOCONV;
    }
}

static size_t hetrd_smem(int nmax, int fp32) {
    return fp32 ? ht_big_offset<float>(nmax) + ht_big_bytes<float>()
                : ht_big_offset<double>(nmax) + ht_big_bytes<double>();
}

int mmf_hetrd_max_n(int fp32) {
    const size_t cs = fp32 ? 8 : 16;
    const size_t fixed = fp32 ? ht_fixed_bytes<float>() + ht_big_bytes<float>()
                              : ht_fixed_bytes<double>() + ht_big_bytes<double>();
    // 64 bytes for the kernel's static shared variables (tensor-core mbarriers, TMEM address) and
    // the 16-byte rounding of the operand region
    return (int)((227 * 1024 - fixed - 64) / (3 * cs));
}

template <class R, int CL, bool TC>
static cudaError_t launch_hetrd(const MmfLaunch& L, void* H, void* Vp, void* Wp, double* dvec,
                                double* evec, void* tau, size_t sm, int* status) {
    typedef typename Cx<R>::T C;
    cudaError_t err = cudaFuncSetAttribute(k_hetrd<R, CL, TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (err != cudaSuccess) return err;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.count * CL);
    cfg.blockDim = dim3(HT_THREADS);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_hetrd<R, CL, TC>, L.desc, L.idx, (C*)H, (C*)Vp, (C*)Wp, dvec, evec,
                              (C*)tau, L.nmax, status);
}

cudaError_t mmf_launch_hetrd(const MmfLaunch& L, void* H, void* Vp, void* Wp, double* dvec,
                             double* evec, void* tau, int fp32, int tc, int* status) {
    if (L.count <= 0) return cudaSuccess;
    if (L.nmax > mmf_hetrd_max_n(fp32)) return cudaErrorInvalidValue;
    const size_t sm = hetrd_smem(L.nmax, fp32);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // two CTAs per system while that still fits the GPU in one wave
    const bool pair = 2 * L.count <= sms;
    if (fp32 && tc)
        return pair ? launch_hetrd<float, 2, true>(L, H, Vp, Wp, dvec, evec, tau, sm, status)
                    : launch_hetrd<float, 1, true>(L, H, Vp, Wp, dvec, evec, tau, sm, status);
    if (fp32)
        return pair ? launch_hetrd<float, 2, false>(L, H, Vp, Wp, dvec, evec, tau, sm, status)
                    : launch_hetrd<float, 1, false>(L, H, Vp, Wp, dvec, evec, tau, sm, status);
    return pair ? launch_hetrd<double, 2, false>(L, H, Vp, Wp, dvec, evec, tau, sm, status)
                : launch_hetrd<double, 1, false>(L, H, Vp, Wp, dvec, evec, tau, sm, status);
}

// ------------------------------------------------------------------ self-test
// `count` seeded Hermitian n x n FP32 matrices (entries uniform in the unit square, full
// mantissas; leading dimension n rounded up to 8) reduced in one launch (two CTAs per system when
// 2 count fits the SMs, else one), with the trailing update on the tensor cores (tc = 1) or the
// FP32 units (tc = 0).  For the first two systems the host applies the stored reflectors to the
// input in FP64, B = P_{n-2}^H ... P_0^H A P_0 ... P_{n-2}, and returns max |B - tridiag(e, d, e)|
// (every entry) and max |A|.  Returns 0, -1 (bad sizes), -4 (CUDA failure) or 1 (a wait gave up).
int mmf_hetrd_selftest_impl(int n, int count, int tc, double* max_err, double* max_ref) {
    if (n < 2 || n > mmf_hetrd_max_n(1) || count < 1 || count > 512 || (int64_t)n * n * count > (1 << 27)) return -1;
    const int ld = (n + 7) & ~7;
    const int64_t mat = (int64_t)n * ld, pan = (int64_t)ld * MMF_NB;
    std::vector<MmfDesc> hd(count);
    std::vector<int> hidx(count);
    for (int s = 0; s < count; ++s) {
        MmfDesc d = {};
        d.n = n;
        d.ld = ld;
        d.D = n;
        d.M = 1;
        d.mat_off = s * mat;
        d.pan_off = s * pan;
        d.vec_off = (int64_t)s * n;
        hd[s] = d;
        hidx[s] = s;
    }
    std::vector<float2> hA((size_t)mat * count, make_float2(0.f, 0.f));
    uint64_t x = 0x9E3779B97F4A7C15ull;
    auto unif = [&x]() {  // xorshift64*, uniform in [-1, 1)
        x ^= x >> 12;
        x ^= x << 25;
        x ^= x >> 27;
        return (double)((x * 0x2545F4914F6CDD1Dull) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
    };
    for (int s = 0; s < count; ++s)
        for (int c = 0; c < n; ++c)
            for (int r = c; r < n; ++r) {
                const float re = (float)unif(), im = r == c ? 0.f : (float)unif();
                hA[s * mat + r + (int64_t)c * ld] = make_float2(re, im);
                hA[s * mat + c + (int64_t)r * ld] = make_float2(re, -im);
            }
    MmfDesc* dd = nullptr;
    int *didx = nullptr, *dst = nullptr;
    float2 *dA = nullptr, *dV = nullptr, *dW = nullptr, *dtau = nullptr;
    double *dD = nullptr, *dE = nullptr;
    int rc = 0;
    cudaStream_t st = nullptr;
    if (cudaStreamCreate(&st) != cudaSuccess) return -4;
    bool ok = cudaMalloc(&dd, sizeof(MmfDesc) * count) == cudaSuccess &&
              cudaMalloc(&didx, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&dst, sizeof(int) * count) == cudaSuccess &&
              cudaMalloc(&dA, sizeof(float2) * mat * count) == cudaSuccess &&
              cudaMalloc(&dV, sizeof(float2) * pan * count) == cudaSuccess &&
              cudaMalloc(&dW, sizeof(float2) * pan * count) == cudaSuccess &&
              cudaMalloc(&dtau, sizeof(float2) * n * count) == cudaSuccess &&
              cudaMalloc(&dD, sizeof(double) * n * count) == cudaSuccess &&
              cudaMalloc(&dE, sizeof(double) * n * count) == cudaSuccess;
    std::vector<double> hD((size_t)n * count), hE((size_t)n * count);
    std::vector<float2> htau((size_t)n * count);
    std::vector<int> hst(count);
    if (ok) {
        ok = cudaMemcpy(dd, hd.data(), sizeof(MmfDesc) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemcpy(didx, hidx.data(), sizeof(int) * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(dst, 0, sizeof(int) * count) == cudaSuccess &&
             cudaMemcpy(dA, hA.data(), sizeof(float2) * mat * count, cudaMemcpyHostToDevice) == cudaSuccess &&
             cudaMemset(dV, 0, sizeof(float2) * pan * count) == cudaSuccess &&
             cudaMemset(dW, 0, sizeof(float2) * pan * count) == cudaSuccess;
        MmfLaunch L = {dd, didx, count, n, st};
        ok = ok && mmf_launch_hetrd(L, dA, dV, dW, dD, dE, dtau, 1, tc, dst) == cudaSuccess &&
             cudaStreamSynchronize(st) == cudaSuccess;
        std::vector<float2> hR((size_t)mat * count);
        ok = ok && cudaMemcpy(hR.data(), dA, sizeof(float2) * mat * count, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(hD.data(), dD, sizeof(double) * n * count, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(hE.data(), dE, sizeof(double) * n * count, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(htau.data(), dtau, sizeof(float2) * n * count, cudaMemcpyDeviceToHost) == cudaSuccess &&
             cudaMemcpy(hst.data(), dst, sizeof(int) * count, cudaMemcpyDeviceToHost) == cudaSuccess;
        if (ok) {
            for (int s = 0; s < count; ++s)
                if (hst[s] != 0) rc = 1;
            double err = 0.0, ref = 0.0;
            std::vector<double2> B((size_t)n * n), v(n), y(n);
            for (int s = 0; s < std::min(count, 2); ++s) {
                const float2* A0 = hA.data() + s * mat;
                const float2* R = hR.data() + s * mat;
                for (int c = 0; c < n; ++c)
                    for (int r = 0; r < n; ++r) {
                        const float2 a = A0[r + (int64_t)c * ld];
                        B[r + (size_t)c * n] = make_double2(a.x, a.y);
                        ref = std::max(ref, std::hypot((double)a.x, (double)a.y));
                    }
                for (int k = 0; k + 1 < n; ++k) {  // B <- P_k^H B P_k, P_k = I - tau v v^H
                    const float2 tf = htau[(size_t)s * n + k];
                    const double tr = tf.x, ti = tf.y;
                    for (int r = 0; r < n; ++r) {
                        if (r <= k) v[r] = make_double2(0.0, 0.0);
                        else if (r == k + 1) v[r] = make_double2(1.0, 0.0);
                        else v[r] = make_double2(R[r + (int64_t)k * ld].x, R[r + (int64_t)k * ld].y);
                    }
                    // B <- B P = B - tau (B v) v^H
                    for (int r = 0; r < n; ++r) {
                        double yr = 0.0, yi = 0.0;
                        for (int c = k + 1; c < n; ++c) {
                            const double2 b = B[r + (size_t)c * n];
                            yr += b.x * v[c].x - b.y * v[c].y;
                            yi += b.x * v[c].y + b.y * v[c].x;
                        }
                        const double ur = tr * yr - ti * yi, ui = tr * yi + ti * yr;  // tau (B v)_r
                        for (int c = k + 1; c < n; ++c) {  // - u conj(v_c)
                            double2& b = B[r + (size_t)c * n];
                            b.x -= ur * v[c].x + ui * v[c].y;
                            b.y -= ui * v[c].x - ur * v[c].y;
                        }
                    }
                    // B <- P^H B = B - conj(tau) v (v^H B)
                    for (int c = 0; c < n; ++c) {
                        double yr = 0.0, yi = 0.0;
                        for (int r = k + 1; r < n; ++r) {
                            const double2 b = B[r + (size_t)c * n];
                            yr += v[r].x * b.x + v[r].y * b.y;
                            yi += v[r].x * b.y - v[r].y * b.x;
                        }
                        const double ur = tr * yr + ti * yi, ui = tr * yi - ti * yr;  // conj(tau) (v^H B)_c
                        for (int r = k + 1; r < n; ++r) {
                            double2& b = B[r + (size_t)c * n];
                            b.x -= v[r].x * ur - v[r].y * ui;
                            b.y -= v[r].x * ui + v[r].y * ur;
                        }
                    }
                }
                for (int c = 0; c < n; ++c)
                    for (int r = 0; r < n; ++r) {
                        double2 t = make_double2(0.0, 0.0);
                        if (r == c) t.x = hD[(size_t)s * n + r];
                        else if (r == c + 1) t.x = hE[(size_t)s * n + c];
                        else if (c == r + 1) t.x = hE[(size_t)s * n + r];
                        const double2 b = B[r + (size_t)c * n];
                        err = std::max(err, std::hypot(b.x - t.x, b.y - t.y));
                    }
            }
            *max_err = err;
            *max_ref = ref;
        }
    }
    if (!ok) rc = -4;
    cudaFree(dd);
    cudaFree(didx);
    cudaFree(dst);
    cudaFree(dA);
    cudaFree(dV);
    cudaFree(dW);
    cudaFree(dtau);
    cudaFree(dD);
    cudaFree(dE);
    cudaStreamDestroy(st);
    return rc;
}
