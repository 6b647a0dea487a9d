// k_hetrd_large.cu -- S2 for one large system: the blocked Householder reduction of k_hetrd.cu
// (same reflectors, same deferred panel updates, same outputs) spread over the whole GPU.
//
// Only the lower triangle is kept (as on the one-CTA path): y = A22 v is a Hermitian product in
// which each lower entry serves its row and (conjugated) its column; a grid of CTAs each owns a
// 128 x 128 block on or below the diagonal and adds its row and column sums into y with atomics.  Per column k (panel position i) the host
// enqueues six launches: (1a) the grid applies the pending panel updates to column k and sums
// |A(r, k)|^2 below the subdiagonal; (1b) one thread forms the reflector; (1c) the grid scales
// the column into v, clears y and sums the short products W^H v, V^H v; (2) the grid forms
// y = A22 v; (3) the grid applies the panel corrections, w = tau y and the partial sums of w^H v;
// (4) the grid finishes w += -(1/2) tau (w^H v) v into W(:, i).  The column's steps are spread
// over the grid because they read the panel (m x 2i entries): one CTA streamed it at a few tens
// of GB/s, as long as the gemv over the whole trailing matrix.  After each panel a grid-wide
// update A -= V W^H + W V^H touches the lower triangle of the trailing matrix.  It stays on the
// FP32 / FP64 units: tens of thousands of small CTAs hide its HBM latency, which a tensor-core version
// with one CTA per SM and one tile in flight did not (7.2 against 5.4 ms per panel at n = 17576).
#include "mmf_internal.h"

#define LG_B 256      // rows per CTA of the column kernels
#define LG_TILE 64    // trailing-update tile

struct LgScalars {     // per-column scalars shared between the launches (device memory)
    double2 tau;       // reflector scalar (in the working precision, widened)
    double2 dot;       // accumulated w^H v
    double2 scale;     // 1 / (alpha - beta): multiplies the column into v
    double xn2;        // accumulated |A(r, k)|^2 over r >= k + 2 (cleared by the reflector kernel)
    double pad;
};
static_assert(sizeof(LgScalars) <= 8 * sizeof(double), "the scalars fit the system's 8-double auxiliary slot");

template <class R>
__device__ __forceinline__ R cta_sum(R v, R* red) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        R s = (threadIdx.x < (int)(blockDim.x >> 5)) ? red[threadIdx.x] : R(0);
        s = warp_sum(s);
        if (threadIdx.x == 0) red[32] = s;
    }
    __syncthreads();
    R r = red[32];
    __syncthreads();
    return r;
}

__device__ __forceinline__ void atomic_add_cx(double2* p, double2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}
__device__ __forceinline__ void atomic_add_cx(float2* p, float2 v) {
    atomicAdd(&p->x, v.x);
    atomicAdd(&p->y, v.y);
}

// (1a) column k = j0 + i over the grid: pending panel updates of rows k .., and the sum of
// |A(r, k)|^2 over r >= k + 2 into sc->xn2
template <class R>
__global__ void __launch_bounds__(LG_B) k_lg_colupd(typename Cx<R>::T* __restrict__ A, int n, int ld, int k, int i,
                                                    const typename Cx<R>::T* __restrict__ V,
                                                    const typename Cx<R>::T* __restrict__ W, LgScalars* sc) {
    typedef typename Cx<R>::T C;
    __shared__ C wk[MMF_NB], vk[MMF_NB];
    __shared__ R red[33];
    const int tid = threadIdx.x;
    if (tid < i) {
        wk[tid] = conj(W[k + (int64_t)tid * ld]);
        vk[tid] = conj(V[k + (int64_t)tid * ld]);
    }
    __syncthreads();
    const int r = k + blockIdx.x * LG_B + tid;
    R part = 0;
    if (r < n) {
        C* pc = A + (int64_t)k * ld + r;
        C x = *pc;
        if (i > 0) {
            C acc = czero<C>(), acc2 = czero<C>();
#pragma unroll 8
            for (int c = 0; c < i; ++c) {
                acc = acc + V[r + (int64_t)c * ld] * wk[c];
                acc2 = acc2 + W[r + (int64_t)c * ld] * vk[c];
            }
            x = x - (acc + acc2);
            *pc = x;
        }
        if (r >= k + 2) part = abs2(x);
    }
    const R sum = cta_sum(part, red);
    if (tid == 0 && sum != R(0)) atomicAdd(&sc->xn2, (double)sum);
}

// (1b) the reflector of column k (one thread), and the cleared sums of the column's later steps
template <class R>
__global__ void k_lg_refl(typename Cx<R>::T* __restrict__ A, int n, int ld, int k, typename Cx<R>::T* __restrict__ xbuf,
                          LgScalars* sc, double* __restrict__ dd, double* __restrict__ ee,
                          typename Cx<R>::T* __restrict__ tau) {
    typedef typename Cx<R>::T C;
    if (threadIdx.x < 2 * MMF_NB) xbuf[threadIdx.x] = czero<C>();
    if (threadIdx.x != 0) return;
    const C* col = A + (int64_t)k * ld;
    dd[k] = (double)col[k].x;
    const R xn2 = (R)sc->xn2;
    sc->xn2 = 0.0;
    if (k == n - 1) return;
    const C alpha = col[k + 1];
    C t, s;
    R beta;
    if (xn2 == R(0) && alpha.y == R(0)) {
        t = czero<C>();
        s = czero<C>();
        beta = alpha.x;
    } else {
        beta = -copysign(sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xn2), alpha.x);
        t = mk((beta - alpha.x) / beta, -alpha.y / beta);
        const C den = mk(alpha.x - beta, alpha.y);
        const R dn = abs2(den);
        s = mk(den.x / dn, -den.y / dn);
    }
    ee[k] = (double)beta;
    tau[k] = t;
    sc->tau = to_c128(t);
    sc->scale = to_c128(s);
    sc->dot = make_double2(0.0, 0.0);
}

// (1c) v from column k over the grid (rows of this CTA): A(r, k) <- v_r below the subdiagonal,
// V(:, i), vbuf, y = 0; then the CTA's parts of x_w = W^H v and x_v = V^H v (warp per product)
template <class R>
__global__ void __launch_bounds__(LG_B) k_lg_vscale(typename Cx<R>::T* __restrict__ A, int n, int ld, int k, int i,
                                                    typename Cx<R>::T* __restrict__ V,
                                                    const typename Cx<R>::T* __restrict__ W,
                                                    typename Cx<R>::T* __restrict__ vbuf,
                                                    typename Cx<R>::T* __restrict__ ybuf,
                                                    typename Cx<R>::T* __restrict__ xbuf, const LgScalars* sc) {
    typedef typename Cx<R>::T C;
    __shared__ C vs[LG_B];
    const int tid = threadIdx.x, r0 = blockIdx.x * LG_B, r = r0 + tid;
    const C scale = from_c128<C>(sc->scale);
    C v = czero<C>();
    if (r < n) {
        if (r == k + 1) {
            v = mk(R(1), R(0));
        } else if (r > k + 1) {
            C* pc = A + (int64_t)k * ld + r;
            v = *pc * scale;
            *pc = v;
        }
        if (r > k) {
            vbuf[r - k - 1] = v;
            ybuf[r - k - 1] = czero<C>();
        }
        V[r + (int64_t)i * ld] = v;
    }
    vs[tid] = v;  // zero at and above row k, and past n
    __syncthreads();
    if (r0 + LG_B <= k + 1) return;  // no row of this CTA lies below row k
    const int lane = tid & 31, warp = tid >> 5;
    for (int task = warp; task < 2 * i; task += LG_B / 32) {
        const int c = task >> 1;
        const C* P = (task & 1) ? V : W;
        C acc = czero<C>();
#pragma unroll
        for (int u = 0; u < LG_B / 32; ++u) {
            const int rr = r0 + lane + 32 * u;
            if (rr > k && rr < n) acc = acc + cmulc(P[rr + (int64_t)c * ld], vs[lane + 32 * u]);
        }
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane == 0) atomic_add_cx(&xbuf[task], acc);  // xbuf[2c] = (W^H v)_c, xbuf[2c+1] = (V^H v)_c
    }
}

// (2) y += A22 v from the lower triangle of A22 = A(k+1:, k+1:): one CTA per 128 x 128 block
// (I, J) with I >= J, numbered along block rows (block b: I = floor((sqrt(8 b + 1) - 1) / 2),
// J = b - I (I + 1) / 2).  Thread (row r, column half h) reads its 64 entries A(r, c) once and
// adds a(r, c) v_c to its row's sum and conj(a(r, c)) v_r to column c's sum (strictly below the
// diagonal; the diagonal entry once, as a real number).  Column sums: a butterfly reduce-scatter
// of 8 columns at a time over the 32 rows of a warp (16 shuffles for 16 values), then shared
// memory over the block's four warps of that half.
#define LG_HB 128
template <class R>
__global__ void __launch_bounds__(256) k_lg_hemv(const typename Cx<R>::T* __restrict__ A, int n, int ld, int k,
                                                 const typename Cx<R>::T* __restrict__ vbuf,
                                                 typename Cx<R>::T* __restrict__ ybuf) {
    typedef typename Cx<R>::T C;
    __shared__ C vr_s[LG_HB], vc_s[LG_HB];
    __shared__ C colsum[4][LG_HB];  // [warp within the half][column]
    const int m = n - k - 1;
    const int bI = (int)((sqrt(8.0 * blockIdx.x + 1.0) - 1.0) * 0.5);
    int I = bI, J = (int)blockIdx.x - bI * (bI + 1) / 2;
    if (J > I) {  // rounding of the square root: the next block row
        J -= I + 1;
        ++I;
    } else if (J < 0) {  // or the previous one
        --I;
        J += I + 1;
    }
    const int r0 = I * LG_HB, c0 = J * LG_HB;
    if (r0 >= m) return;
    const int tid = threadIdx.x;
    if (tid < LG_HB) {
        vr_s[tid] = (r0 + tid < m) ? vbuf[r0 + tid] : czero<C>();
        vc_s[tid] = (c0 + tid < m) ? vbuf[c0 + tid] : czero<C>();
    }
    __syncthreads();
    const int rl = tid & (LG_HB - 1), h = tid >> 7, lane = tid & 31, wq = (tid >> 5) & 3;
    const int r = r0 + rl;
    const bool rok = r < m;
    const C vr = vr_s[rl];
    const C* a = A + (k + 1 + (rok ? r : 0)) + (int64_t)(k + 1 + c0 + 64 * h) * ld;
    C acc = czero<C>();
    for (int q0 = 0; q0 < 64; q0 += 8) {
        C av[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int cl = 64 * h + q0 + u, c = c0 + cl;
            const bool ok = rok && c < m && (I > J || c <= r);
            av[u] = ok ? a[(int64_t)(q0 + u) * ld] : czero<C>();
        }
        R cv[16];  // column parts of the 8 columns (Re, Im), strictly below the diagonal
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int cl = 64 * h + q0 + u, c = c0 + cl;
            const bool diag = (I == J) && c == r;
            const C aa = diag ? mk(av[u].x, R(0)) : av[u];
            acc = acc + aa * vc_s[cl];
            const C cp = diag ? czero<C>() : cmulc(av[u], vr);
            cv[2 * u] = cp.x;
            cv[2 * u + 1] = cp.y;
        }
        // the 16 sums over the warp's 32 rows by a butterfly reduce-scatter: after the rounds
        // with lane offsets 16, 8, 4, 2 lane L holds value (L >> 1) & 15 summed over 16 lanes,
        // and the last round adds its partner's
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const bool hi = lane & 16;
            const R keep = hi ? cv[t + 8] : cv[t], send = hi ? cv[t] : cv[t + 8];
            cv[t] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const bool hi = lane & 8;
            const R keep = hi ? cv[t + 4] : cv[t], send = hi ? cv[t] : cv[t + 4];
            cv[t] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const bool hi = lane & 4;
            const R keep = hi ? cv[t + 2] : cv[t], send = hi ? cv[t] : cv[t + 2];
            cv[t] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
        {
            const bool hi = lane & 2;
            const R keep = hi ? cv[1] : cv[0], send = hi ? cv[0] : cv[1];
            cv[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
        }
        cv[0] += __shfl_xor_sync(0xffffffffu, cv[0], 1);
        if ((lane & 1) == 0) {
            const int idx = (lane >> 1) & 15;  // column q0 + idx / 2, Re (idx even) or Im
            reinterpret_cast<R*>(&colsum[wq][64 * h + q0 + (idx >> 1)])[idx & 1] = cv[0];
        }
    }
    if (rok) atomic_add_cx(&ybuf[r], acc);
    __syncthreads();
    if (tid < LG_HB) {
        const int c = c0 + tid;
        if (c < m) {
            // the four warps of the column's half: rows 0..127 of the block
            C s = colsum[0][tid];
            for (int w = 1; w < 4; ++w) s = s + colsum[w][tid];
            atomic_add_cx(&ybuf[c], s);
        }
    }
}

// (3) y -= V x_w + W x_v;  w = tau y (into W(:, i));  dot += w^H v
template <class R>
__global__ void __launch_bounds__(LG_B) k_lg_w(int n, int ld, int k, int i,
                                               const typename Cx<R>::T* __restrict__ V,
                                               typename Cx<R>::T* __restrict__ W,
                                               const typename Cx<R>::T* __restrict__ vbuf,
                                               const typename Cx<R>::T* __restrict__ ybuf,
                                               const typename Cx<R>::T* __restrict__ xbuf, LgScalars* sc) {
    typedef typename Cx<R>::T C;
    __shared__ C xs[2 * MMF_NB];
    __shared__ R red[33];
    const int m = n - k - 1;
    if (threadIdx.x < 2 * i) xs[threadIdx.x] = xbuf[threadIdx.x];
    __syncthreads();
    const C tk = from_c128<C>(sc->tau);
    const int rp = blockIdx.x * LG_B + threadIdx.x;
    C dpart = czero<C>();
    if (rp < m) {
        C y = ybuf[rp];
        for (int c = 0; c < i; ++c)
            y = y - V[(k + 1 + rp) + (int64_t)c * ld] * xs[2 * c] - W[(k + 1 + rp) + (int64_t)c * ld] * xs[2 * c + 1];
        const C w = tk * y;
        W[(k + 1 + rp) + (int64_t)i * ld] = w;
        dpart = cmulc(w, vbuf[rp]);
    }
    const R dx = cta_sum(dpart.x, red), dy = cta_sum(dpart.y, red);
    if (threadIdx.x == 0) atomic_add_cx(&sc->dot, make_double2((double)dx, (double)dy));
}

// (4) W(:, i) = w - (1/2) tau (w^H v) v below k, 0 above
template <class R>
__global__ void __launch_bounds__(LG_B) k_lg_w2(int n, int ld, int k, int i, typename Cx<R>::T* __restrict__ W,
                                                const typename Cx<R>::T* __restrict__ vbuf, const LgScalars* sc) {
    typedef typename Cx<R>::T C;
    const int r = blockIdx.x * LG_B + threadIdx.x;
    if (r >= n) return;
    if (r <= k) {
        W[r + (int64_t)i * ld] = czero<C>();
        return;
    }
    const C tk = from_c128<C>(sc->tau);
    const C alpha2 = R(-0.5) * (tk * from_c128<C>(sc->dot));
    W[r + (int64_t)i * ld] = W[r + (int64_t)i * ld] + alpha2 * vbuf[r - k - 1];
}

// trailing update of the lower triangle: A(c0:, c0:) -= V W^H + W V^H, 64 x 64 tiles on and below
// the diagonal (the diagonal tiles masked to r >= c), the panel's columns staged 8 at a time
#define LG_KC 8
template <class R>
__global__ void __launch_bounds__(256) k_lg_her2k(typename Cx<R>::T* __restrict__ A, int n, int ld, int c0, int nb,
                                                  const typename Cx<R>::T* __restrict__ V,
                                                  const typename Cx<R>::T* __restrict__ W) {
    typedef typename Cx<R>::T C;
    __shared__ C tVr[LG_KC][LG_TILE], tWr[LG_KC][LG_TILE], tVc[LG_KC][LG_TILE], tWc[LG_KC][LG_TILE];
    const int rbase = c0 + blockIdx.x * LG_TILE, cbase = c0 + blockIdx.y * LG_TILE;
    if (rbase >= n || cbase >= n || blockIdx.x < blockIdx.y) return;
    const int rr = threadIdx.x & 63, cg = threadIdx.x >> 6;  // 4 column groups, 16 columns each
    C acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = czero<C>();
    for (int p0 = 0; p0 < nb; p0 += LG_KC) {
        __syncthreads();
        for (int e = threadIdx.x; e < LG_KC * LG_TILE; e += 256) {
            const int p = e / LG_TILE, q = e - p * LG_TILE;
            const int r = rbase + q, c = cbase + q;
            const bool pv = p0 + p < nb;
            tVr[p][q] = (pv && r < n) ? V[r + (int64_t)(p0 + p) * ld] : czero<C>();
            tWr[p][q] = (pv && r < n) ? W[r + (int64_t)(p0 + p) * ld] : czero<C>();
            tVc[p][q] = (pv && c < n) ? conj(V[c + (int64_t)(p0 + p) * ld]) : czero<C>();
            tWc[p][q] = (pv && c < n) ? conj(W[c + (int64_t)(p0 + p) * ld]) : czero<C>();
        }
        __syncthreads();
#pragma unroll
        for (int p = 0; p < LG_KC; ++p) {
            const C a = tVr[p][rr], b = tWr[p][rr];
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int cc = cg + 4 * q;
                acc[q] = acc[q] + a * tWc[p][cc] + b * tVc[p][cc];
            }
        }
    }
    const int r = rbase + rr;
    if (r < n)
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const int c = cbase + cg + 4 * q;
            if (c < n && r >= c) {
                C* pa = A + r + (int64_t)c * ld;
                *pa = *pa - acc[q];
            }
        }
}

template <class R>
static cudaError_t run_large(typename Cx<R>::T* A, int n, int ld, typename Cx<R>::T* V, typename Cx<R>::T* W,
                             typename Cx<R>::T* work, LgScalars* sc, double* dd, double* ee,
                             typename Cx<R>::T* tau, cudaStream_t st) {
    typedef typename Cx<R>::T C;
    C* vbuf = work;
    C* ybuf = work + n;
    C* xbuf = work + 2 * (size_t)n;
    cudaError_t e0 = cudaMemsetAsync(sc, 0, sizeof(LgScalars), st);
    if (e0 != cudaSuccess) return e0;
    for (int j0 = 0; j0 < n; j0 += MMF_NB) {
        const int nb = min(MMF_NB, n - j0);
        for (int i = 0; i < nb; ++i) {
            const int k = j0 + i;
            k_lg_colupd<R><<<(n - k + LG_B - 1) / LG_B, LG_B, 0, st>>>(A, n, ld, k, i, V, W, sc);
            k_lg_refl<R><<<1, 2 * MMF_NB, 0, st>>>(A, n, ld, k, xbuf, sc, dd, ee, tau);
            if (k == n - 1) break;
            k_lg_vscale<R><<<(n + LG_B - 1) / LG_B, LG_B, 0, st>>>(A, n, ld, k, i, V, W, vbuf, ybuf, xbuf, sc);
            const int m = n - k - 1;
            const int g = (m + LG_B - 1) / LG_B;
            const int gb = (m + LG_HB - 1) / LG_HB;
            k_lg_hemv<R><<<gb * (gb + 1) / 2, 256, 0, st>>>(A, n, ld, k, vbuf, ybuf);
            k_lg_w<R><<<g, LG_B, 0, st>>>(n, ld, k, i, V, W, vbuf, ybuf, xbuf, sc);
            k_lg_w2<R><<<(n + LG_B - 1) / LG_B, LG_B, 0, st>>>(n, ld, k, i, W, vbuf, sc);
        }
        const int c0 = j0 + nb;
        if (c0 < n) {
            const int g = (n - c0 + LG_TILE - 1) / LG_TILE;
            k_lg_her2k<R><<<dim3(g, g), 256, 0, st>>>(A, n, ld, c0, nb, V, W);
        }
    }
    return cudaGetLastError();
}

// One large system (host-side descriptor copy `d`, device pointers into the batch pools).
// work: 3 n + 2 NB complex elements of the working precision; sc: one LgScalars.
cudaError_t mmf_launch_hetrd_large(const MmfDesc& d, void* H, void* Vp, void* Wp, double* dvec, double* evec,
                                   void* tau, void* work, void* sc, int fp32, cudaStream_t st) {
    if (fp32)
        return run_large<float>((float2*)H + d.mat_off, d.n, d.ld, (float2*)Vp + d.pan_off, (float2*)Wp + d.pan_off,
                                (float2*)work, (LgScalars*)sc, dvec + d.vec_off, evec + d.vec_off,
                                (float2*)tau + d.vec_off, st);
    return run_large<double>((double2*)H + d.mat_off, d.n, d.ld, (double2*)Vp + d.pan_off, (double2*)Wp + d.pan_off,
                             (double2*)work, (LgScalars*)sc, dvec + d.vec_off, evec + d.vec_off,
                             (double2*)tau + d.vec_off, st);
}

size_t mmf_hetrd_large_scalars_bytes() { return sizeof(LgScalars); }
