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

#include "mmf_internal.h"

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
template <class R>
__host__ __device__ constexpr size_t ht_big_bytes() {
    return sizeof(R) == 4 ? (size_t)(HT_THREADS / 32) * 2 * HT_STAGE_ELEMS * sizeof(typename Cx<R>::T)
                          : (size_t)4 * MMF_NB * HT_TILE * sizeof(typename Cx<R>::T);
}

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

template <class R, int CL>
__global__ void __launch_bounds__(HT_THREADS, 1)
k_hetrd(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
        typename Cx<R>::T* __restrict__ H, typename Cx<R>::T* __restrict__ Vpool,
        typename Cx<R>::T* __restrict__ Wpool, double* __restrict__ dvec,
        double* __restrict__ evec, typename Cx<R>::T* __restrict__ taupool, int nmax) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
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
        if (c0 < n) {
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
}

static size_t hetrd_smem(int nmax, int fp32) {
    return fp32 ? ht_big_offset<float>(nmax) + ht_big_bytes<float>()
                : ht_big_offset<double>(nmax) + ht_big_bytes<double>();
}

int mmf_hetrd_max_n(int fp32) {
    const size_t cs = fp32 ? 8 : 16;
    const size_t fixed = fp32 ? ht_fixed_bytes<float>() + ht_big_bytes<float>()
                              : ht_fixed_bytes<double>() + ht_big_bytes<double>();
    return (int)((227 * 1024 - fixed - 16) / (3 * cs));
}

template <class R, int CL>
static cudaError_t launch_hetrd(const MmfLaunch& L, void* H, void* Vp, void* Wp, double* dvec,
                                double* evec, void* tau, size_t sm) {
    typedef typename Cx<R>::T C;
    cudaError_t err = cudaFuncSetAttribute(k_hetrd<R, CL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
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
    return cudaLaunchKernelEx(&cfg, k_hetrd<R, CL>, L.desc, L.idx, (C*)H, (C*)Vp, (C*)Wp, dvec, evec,
                              (C*)tau, L.nmax);
}

cudaError_t mmf_launch_hetrd(const MmfLaunch& L, void* H, void* Vp, void* Wp, double* dvec,
                             double* evec, void* tau, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    if (L.nmax > mmf_hetrd_max_n(fp32)) return cudaErrorInvalidValue;
    const size_t sm = hetrd_smem(L.nmax, fp32);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // two CTAs per system while that still fits the GPU in one wave
    const bool pair = 2 * L.count <= sms;
    if (fp32)
        return pair ? launch_hetrd<float, 2>(L, H, Vp, Wp, dvec, evec, tau, sm)
                    : launch_hetrd<float, 1>(L, H, Vp, Wp, dvec, evec, tau, sm);
    return pair ? launch_hetrd<double, 2>(L, H, Vp, Wp, dvec, evec, tau, sm)
                : launch_hetrd<double, 1>(L, H, Vp, Wp, dvec, evec, tau, sm);
}
