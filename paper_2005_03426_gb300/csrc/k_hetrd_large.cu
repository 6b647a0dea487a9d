// k_hetrd_large.cu -- S2 for one large system: the blocked Householder reduction of k_hetrd.cu
// (same reflectors, same deferred panel updates, same outputs) spread over the whole GPU.
//
// The matrix is kept in full Hermitian storage so that y = A22 v is a plain matrix-vector
// product: a grid of CTAs each owns a 256 x 256 block of the trailing matrix and adds its
// rows' partial sums into y with one atomic per row.  Per column k (panel position i) the host
// enqueues four launches: (1) one CTA applies the pending panel updates to column k, forms the
// reflector and the short products W^H v, V^H v and clears y; (2) the grid forms y = A22 v;
// (3) the grid applies the panel corrections, w = tau y and the partial sums of w^H v;
// (4) the grid finishes w += -(1/2) tau (w^H v) v into W(:, i).  After each panel a grid-wide
// update A -= V W^H + W V^H touches both triangles of the trailing matrix.
#include "mmf_internal.h"

#define LG_T 1024     // threads of the one-CTA column kernel
#define LG_B 256      // gemv block (rows and columns) and threads per gemv CTA
#define LG_TILE 64    // trailing-update tile

struct LgScalars {     // per-column scalars shared between the launches (device memory)
    double2 tau;       // reflector scalar (in the working precision, widened)
    double2 dot;       // accumulated w^H v
};

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

// (1) column k = j0 + i: pending updates, reflector, W^H v and V^H v, y = 0
template <class R>
__global__ void __launch_bounds__(LG_T) k_lg_col(typename Cx<R>::T* __restrict__ A, int n, int ld, int k, int i,
                                                 typename Cx<R>::T* __restrict__ V,
                                                 typename Cx<R>::T* __restrict__ W,
                                                 typename Cx<R>::T* __restrict__ vbuf,
                                                 typename Cx<R>::T* __restrict__ ybuf,
                                                 typename Cx<R>::T* __restrict__ xbuf, LgScalars* sc,
                                                 double* __restrict__ dd, double* __restrict__ ee,
                                                 typename Cx<R>::T* __restrict__ tau) {
    typedef typename Cx<R>::T C;
    __shared__ C wk[MMF_NB], vk[MMF_NB];
    __shared__ R red[33];
    __shared__ C scs[2];
    const int tid = threadIdx.x;
    if (tid < i) {
        wk[tid] = conj(W[k + (int64_t)tid * ld]);
        vk[tid] = conj(V[k + (int64_t)tid * ld]);
    }
    __syncthreads();
    C* col = A + (int64_t)k * ld;
    if (i > 0)
        for (int r = k + tid; r < n; r += LG_T) {
            C acc = czero<C>();
            for (int c = 0; c < i; ++c) acc = acc + V[r + (int64_t)c * ld] * wk[c] + W[r + (int64_t)c * ld] * vk[c];
            col[r] = col[r] - acc;
        }
    __syncthreads();
    if (tid == 0) dd[k] = (double)col[k].x;
    if (k == n - 1) return;
    const int m = n - k - 1;
    R part = 0;
    for (int r = k + 2 + tid; r < n; r += LG_T) part += abs2(col[r]);
    const R xn2 = cta_sum(part, red);
    if (tid == 0) {
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
        scs[0] = t;
        scs[1] = s;
        sc->tau = to_c128(t);
        sc->dot = make_double2(0.0, 0.0);
    }
    __syncthreads();
    const C scale = scs[1];
    for (int r = tid; r < n; r += LG_T) {
        C v;
        if (r <= k) v = czero<C>();
        else if (r == k + 1) v = mk(R(1), R(0));
        else {
            v = col[r] * scale;
            col[r] = v;
        }
        if (r > k) {
            vbuf[r - k - 1] = v;
            ybuf[r - k - 1] = czero<C>();
        }
        V[r + (int64_t)i * ld] = v;
    }
    __syncthreads();
    // x_w = W^H v, x_v = V^H v over rows k+1.. (one warp per product)
    const int lane = tid & 31, warp = tid >> 5;
    for (int task = warp; task < 2 * i; task += LG_T / 32) {
        const int c = task >> 1;
        const C* P = (task & 1) ? V : W;
        C acc = czero<C>();
        for (int rp = lane; rp < m; rp += 32) acc = acc + cmulc(P[(k + 1 + rp) + (int64_t)c * ld], vbuf[rp]);
        acc.x = warp_sum(acc.x);
        acc.y = warp_sum(acc.y);
        if (lane == 0) xbuf[task] = acc;  // xbuf[2c] = (W^H v)_c, xbuf[2c+1] = (V^H v)_c
    }
}

// (2) y += A22 v over one 256 x 256 block (rows and columns of A22 = A(k+1:, k+1:))
template <class R>
__global__ void __launch_bounds__(LG_B) k_lg_gemv(const typename Cx<R>::T* __restrict__ A, int n, int ld, int k,
                                                  const typename Cx<R>::T* __restrict__ vbuf,
                                                  typename Cx<R>::T* __restrict__ ybuf) {
    typedef typename Cx<R>::T C;
    __shared__ C vs[LG_B];
    const int m = n - k - 1;
    const int r0 = blockIdx.x * LG_B, c0 = blockIdx.y * LG_B;
    if (r0 >= m || c0 >= m) return;
    const int nc = min(LG_B, m - c0);
    if (threadIdx.x < nc) vs[threadIdx.x] = vbuf[c0 + threadIdx.x];
    __syncthreads();
    const int r = r0 + threadIdx.x;
    if (r >= m) return;
    const C* a = A + (k + 1 + r) + (int64_t)(k + 1 + c0) * ld;
    C acc = czero<C>();
#pragma unroll 8
    for (int c = 0; c < nc; ++c) acc = acc + a[(int64_t)c * ld] * vs[c];
    atomic_add_cx(&ybuf[r], acc);
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

// trailing update of both triangles: A(c0:, c0:) -= V W^H + W V^H, 64 x 64 tiles, the panel's
// columns staged 8 at a time
#define LG_KC 8
template <class R>
__global__ void __launch_bounds__(256) k_lg_her2k(typename Cx<R>::T* __restrict__ A, int n, int ld, int c0, int nb,
                                                  const typename Cx<R>::T* __restrict__ V,
                                                  const typename Cx<R>::T* __restrict__ W) {
    typedef typename Cx<R>::T C;
    __shared__ C tVr[LG_KC][LG_TILE], tWr[LG_KC][LG_TILE], tVc[LG_KC][LG_TILE], tWc[LG_KC][LG_TILE];
    const int rbase = c0 + blockIdx.x * LG_TILE, cbase = c0 + blockIdx.y * LG_TILE;
    if (rbase >= n || cbase >= n) return;
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
            if (c < n) {
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
    for (int j0 = 0; j0 < n; j0 += MMF_NB) {
        const int nb = min(MMF_NB, n - j0);
        for (int i = 0; i < nb; ++i) {
            const int k = j0 + i;
            k_lg_col<R><<<1, LG_T, 0, st>>>(A, n, ld, k, i, V, W, vbuf, ybuf, xbuf, sc, dd, ee, tau);
            if (k == n - 1) break;
            const int m = n - k - 1;
            const int g = (m + LG_B - 1) / LG_B;
            k_lg_gemv<R><<<dim3(g, g), LG_B, 0, st>>>(A, n, ld, k, vbuf, ybuf);
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
