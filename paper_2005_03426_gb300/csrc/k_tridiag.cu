// k_tridiag.cu -- S4: eigenpairs of the real symmetric tridiagonal T = tridiag(e, d, e), in FP64
// (the FP64 path) or in FP32 (the mixed path, whose T comes from an FP32 reduction and whose
// eigenpairs are refined afterwards, so FP32 accuracy here loses nothing).
//
// Eigenvalues by Sturm-sequence bisection (Givens 1954; Barth, Martin & Wilkinson 1967):
// count(x) = number of sign changes of the leading principal minors of T - x I (a division-
// free three-term recurrence).  One thread per eigenvalue, each bracketing its own index
// inside the Gershgorin interval until the bracket is below max(2 eps max(|lo|,|hi|), tol |T|)
// (tol = eps of the working precision).  The FP32 solver first scales T by the power of two that
// brings ||T|| to at most 1 (exact), so that the recurrence grows by at most a factor 3 a step.
//
// Eigenvectors by inverse iteration (Wilkinson 1965): (T - lambda I) y = b solved by
// Gaussian elimination with partial pivoting on the tridiagonal band, a fixed number of
// iterations (3) from a hashed start vector.  Eigenvalues closer than ortol = 1e-4 ||T||_1 form a
// cluster (LAPACK's stein takes 1e-3, which at n ~ 2e4 would chain the whole spectrum).  FP64:
// one thread handles a whole cluster in ascending order and orthogonalises each iterate against
// the cluster's earlier vectors (modified Gram-Schmidt), as LAPACK's stein does.  FP32 (followed
// by the refinement): every vector is iterated on its own thread, and each cluster is then
// orthonormalised by one CTA (classical Gram-Schmidt twice per column, in contiguous scratch
// columns), which keeps the serial work per thread at O(n) even where clusters are long.
// Y is written row-major: Y[i * n + k] = component i of eigenvector k.
#include "mmf_internal.h"


__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

#define TRI_CMAX 64  // dot products formed per barrier in the cluster orthonormalisation

// FP32 solver work layout inside a system's slot of 3 n^2 doubles (24 n^2 bytes): from the first
// 16-byte boundary, the packed factors (n^2 float4), the iterate (n^2 floats), then (at an even
// float offset) the scaled (d_i, e_{i-1}^2) pairs and the scaled e_i (3 n floats).  Needs n >= 4.
__device__ __forceinline__ float* tri_f32_base(const float* fwork, const MmfDesc& d) {
    const uintptr_t p = (uintptr_t)(fwork + 6 * d.sq_off);
    return (float*)((p + 15) & ~(uintptr_t)15);
}
__device__ __forceinline__ float2* tri_f32_de2(const float* fwork, const MmfDesc& d) {
    const int64_t nn = (int64_t)d.n * d.n;
    return (float2*)(tri_f32_base(fwork, d) + 5 * nn + (nn & 1));
}

// per system: gl, gu, pivmin, tnorm
__global__ void k_tri_prep(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                           const double* __restrict__ dvec, const double* __restrict__ evec,
                           double* __restrict__ aux, double* __restrict__ e2vec,
                           float* __restrict__ fwork) {
    __shared__ double red[4][32];
    __shared__ double scale_sh;
    const int sid = idx[blockIdx.x];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const double* dd = dvec + d.vec_off;
    const double* ee = evec + d.vec_off;
    double gl = 1e300, gu = -1e300, e2max = 0.0, tn = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double el = (i > 0) ? fabs(ee[i - 1]) : 0.0, er = (i < n - 1) ? fabs(ee[i]) : 0.0;
        gl = fmin(gl, dd[i] - el - er);
        gu = fmax(gu, dd[i] + el + er);
        tn = fmax(tn, fabs(dd[i]) + el + er);
        if (i < n - 1) {
            e2max = fmax(e2max, ee[i] * ee[i]);
            e2vec[d.vec_off + i] = ee[i] * ee[i];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        gl = fmin(gl, __shfl_xor_sync(0xffffffffu, gl, o));
        gu = fmax(gu, __shfl_xor_sync(0xffffffffu, gu, o));
        tn = fmax(tn, __shfl_xor_sync(0xffffffffu, tn, o));
        e2max = fmax(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[0][w] = gl; red[1][w] = gu; red[2][w] = tn; red[3][w] = e2max; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            gl = fmin(gl, red[0][k]); gu = fmax(gu, red[1][k]);
            tn = fmax(tn, red[2][k]); e2max = fmax(e2max, red[3][k]);
        }
        const double eps = 2.220446049250313e-16;
        double pad = 2.0 * eps * fmax(fabs(gl), fabs(gu)) * n + 1e-300;
        aux[8 * sid + 0] = gl - pad;
        aux[8 * sid + 1] = gu + pad;
        aux[8 * sid + 2] = 2.2250738585072014e-308 * fmax(1.0, e2max);  // pivmin
        aux[8 * sid + 3] = tn;
        // FP32 solver: T scaled by s = 2^-k with ||T|| s <= 1
        int ex = 0;
        if (tn > 0.0) frexp(tn, &ex);
        const double sc = ldexp(1.0, -ex);
        aux[8 * sid + 4] = sc;
        scale_sh = sc;
    }
    if (fwork == nullptr) return;
    __syncthreads();
    // scaled FP32 copies after the 5 n^2 floats of the inverse-iteration arrays:
    // (d_i s, e_{i-1}^2 s^2) pairs, then e_i s
    const double sc = scale_sh;
    float2* de2 = tri_f32_de2(fwork, d);
    float* ef = (float*)(de2 + n);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double el = (i > 0) ? ee[i - 1] * sc : 0.0;
        de2[i] = make_float2((float)(dd[i] * sc), (float)(el * el));
        ef[i] = (i < n - 1) ? (float)(ee[i] * sc) : 0.0f;
    }
}

template <class R> struct TriP;
template <> struct TriP<double> {
    static __device__ __forceinline__ double eps() { return 2.220446049250313e-16; }
    static __device__ __forceinline__ double tiny() { return 1e-300; }
    static constexpr double ortol = 1e-4;
    static constexpr int rescale_mask = 15;
};
template <> struct TriP<float> {
    static __device__ __forceinline__ float eps() { return 5.9604645e-8f; }
    static __device__ __forceinline__ float tiny() { return 1e-37f; }
    static constexpr float ortol = 1e-4f;
    static constexpr int rescale_mask = 7;
};

// Power of two 2^-e with e the exponent of v (v > 0 finite), so that v 2^-e lies in [0.5, 1).
__device__ __forceinline__ double pow2_below(double v) {
    int ex;
    frexp(v, &ex);
    return ldexp(1.0, -ex);
}
__device__ __forceinline__ float pow2_below(float v) {
    // exponent field of a normal float; subnormal or zero v takes the scale 2^126
    const int be = (__float_as_int(v) >> 23) & 0xff;
    const int e = be == 0 ? -125 : be - 126;
    const int se = 127 - e;
    return __int_as_float((se < 1 ? 1 : (se > 254 ? 254 : se)) << 23);
}

// Sturm count by the three-term recurrence of the leading principal minors,
//   p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1},
// counting sign changes (= eigenvalues below x); an exact zero takes the sign opposite to its
// predecessor (a negative pivot, as in the ratio form).  Every 16 (FP64) or 8 (FP32) steps the
// pair (p_i, p_{i-1}) is rescaled by the power of two that brings the larger of the two below
// 1, which changes no sign; with ||T|| <= 1 (FP32) a step grows the pair by at most 3, and in
// FP64 the exponent range leaves room for 16 steps at any ||T|| the workloads produce.
// de2[i] = (d_i, e_{i-1}^2) with e_{-1} = 0.
template <class R, class R2>
__device__ __forceinline__ int sturm_count(const R2* __restrict__ de2, int n, R x) {
    int cnt = 0;
    R pm = R(1), p = de2[0].x - x;
    if (p == R(0)) p = -TriP<R>::tiny();
    cnt += (p < R(0));
    for (int i = 1; i < n; ++i) {
        const R2 v = de2[i];
        R pn = fma(v.x - x, p, -v.y * pm);
        if (pn == R(0)) pn = (p < R(0)) ? TriP<R>::tiny() : -TriP<R>::tiny();
        cnt += ((pn < R(0)) != (p < R(0)));
        pm = p;
        p = pn;
        if ((i & TriP<R>::rescale_mask) == 0) {
            const R sc = pow2_below(fmax(fabs(p), fabs(pm)));
            p *= sc;
            pm *= sc;
        }
    }
    return cnt;
}

// FP64 solver input: d and e^2 read from their own arrays.
struct De2View {
    const double* d;
    const double* e2;
    __device__ __forceinline__ double2 operator[](int i) const {
        return make_double2(d[i], i > 0 ? e2[i - 1] : 0.0);
    }
};
__device__ __forceinline__ int sturm_count(const De2View& v, int n, double x) {
    int cnt = 0;
    double pm = 1.0, p = v.d[0] - x;
    if (p == 0.0) p = -1e-300;
    cnt += (p < 0.0);
    for (int i = 1; i < n; ++i) {
        double pn = fma(v.d[i] - x, p, -v.e2[i - 1] * pm);
        if (pn == 0.0) pn = (p < 0.0) ? 1e-300 : -1e-300;
        cnt += ((pn < 0.0) != (p < 0.0));
        pm = p;
        p = pn;
        if ((i & 15) == 0) {
            const double sc = pow2_below(fmax(fabs(p), fabs(pm)));
            p *= sc;
            pm *= sc;
        }
    }
    return cnt;
}

// Per-system views of the solver's inputs in its working precision.
template <class R> struct TriIn;
template <> struct TriIn<double> {
    const double* d;
    const double* e;
    De2View de2;
    double scale;
    __device__ TriIn(const MmfDesc& ds, const double* dvec, const double* evec, const double* e2vec,
                     const double*, const float*) {
        d = dvec + ds.vec_off;
        e = evec + ds.vec_off;
        de2.d = d;
        de2.e2 = e2vec + ds.vec_off;
        scale = 1.0;
    }
    __device__ __forceinline__ double dv(int i) const { return d[i]; }
    __device__ __forceinline__ double ev(int i) const { return e[i]; }
};
template <> struct TriIn<float> {
    const float2* de2;
    const float* e;
    double scale;
    __device__ TriIn(const MmfDesc& ds, const double*, const double*, const double*, const double* aux_sys,
                     const float* fwork) {
        const int n = ds.n;
        de2 = tri_f32_de2(fwork, ds);
        e = (const float*)(de2 + n);
        scale = aux_sys[4];
    }
    __device__ __forceinline__ float dv(int i) const { return de2[i].x; }
    __device__ __forceinline__ float ev(int i) const { return e[i]; }
};

template <class R>
__global__ void __launch_bounds__(128) k_bisect(const MmfDesc* __restrict__ descs,
                                                const int* __restrict__ idx,
                                                const double* __restrict__ dvec,
                                                const double* __restrict__ e2vec,
                                                const double* __restrict__ aux,
                                                const float* __restrict__ fwork,
                                                double* __restrict__ Eout,
                                                int* __restrict__ status) {
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const TriIn<R> in(d, dvec, dvec, e2vec, aux + 8 * sid, fwork);
    const double sc = in.scale;
    // bracket and tolerances in the working precision (scaled for FP32; rounded outwards)
    R lo, hi, pivmin, tn;
    if (sizeof(R) == 4) {
        lo = __double2float_rd(aux[8 * sid] * sc);
        hi = __double2float_ru(aux[8 * sid + 1] * sc);
        pivmin = R(1.1754944e-38);  // e^2 s^2 <= 1 after scaling
        tn = R(aux[8 * sid + 3] * sc);
    } else {
        lo = R(aux[8 * sid]);
        hi = R(aux[8 * sid + 1]);
        pivmin = R(aux[8 * sid + 2]);
        tn = R(aux[8 * sid + 3]);
    }
    const R eps = TriP<R>::eps();
    int it = 0;
    for (; it < 200; ++it) {
        R tol = fmax(R(2) * eps * fmax(fabs(lo), fabs(hi)), eps * tn) + pivmin;
        if (hi - lo <= tol) break;
        R mid = R(0.5) * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(in.de2, n, mid) <= k) lo = mid;
        else hi = mid;
    }
    Eout[d.vec_off + k] = (0.5 * ((double)lo + (double)hi)) / sc;
    if (it >= 200) status[sid] = MMF_ST_NOCONV;
}

// Quotient for the elimination: correctly rounded in FP64; in FP32 the fast reciprocal-based
// quotient (2 ulp), whose denominators here stay far below 2^126 because ||T|| s <= 1.
__device__ __forceinline__ double tdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float tdiv(float a, float b) { return __fdividef(a, b); }

template <class R>
__device__ __forceinline__ R hash_unit(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (R)((double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// Solve (T - lam I) y = y in place; u0/u1/u2 are the (strided) U factor arrays.
#define TRI_PF 8   // steps whose loads are issued ahead of the recurrence (latency hiding)

// (T - lam I) y = b by Gaussian elimination with partial pivoting on the band; the factors go to
// u0, u1, u2 (row stride s), the loads of each TRI_PF steps are issued before their recurrence.
template <class R, class In>
__device__ void tri_solve(const In& in, int n, R lam, R pivtiny, R* y, R* u0, R* u1, R* u2, int64_t s) {
    R p = in.dv(0) - lam, q = (n > 1) ? in.ev(0) : R(0), r = R(0), rb = y[0];
    for (int i0 = 0; i0 < n - 1; i0 += TRI_PF) {
        R av[TRI_PF], dv[TRI_PF], cv[TRI_PF], b1v[TRI_PF];
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 + u;
            const bool ok = i < n - 1;
            av[u] = ok ? in.ev(i) : R(0);
            dv[u] = ok ? in.dv(i + 1) : R(0);
            cv[u] = (i + 1 < n - 1) ? in.ev(i + 1) : R(0);
            b1v[u] = ok ? y[(int64_t)(i + 1) * s] : R(0);
        }
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 + u;
            if (i >= n - 1) break;
            const R a = av[u], bb = dv[u] - lam, cc = cv[u], b1 = b1v[u];
            if (fabs(a) <= fabs(p)) {
                if (p == R(0)) p = pivtiny;
                const R l = tdiv(a, p);
                u0[(int64_t)i * s] = p; u1[(int64_t)i * s] = q; u2[(int64_t)i * s] = r;
                y[(int64_t)i * s] = rb;
                p = bb - l * q; q = cc - l * r; r = R(0); rb = b1 - l * rb;
            } else {
                const R l = tdiv(p, a);
                u0[(int64_t)i * s] = a; u1[(int64_t)i * s] = bb; u2[(int64_t)i * s] = cc;
                y[(int64_t)i * s] = b1;
                const R np = q - l * bb, nq = r - l * cc, nrb = rb - l * b1;
                p = np; q = nq; r = R(0); rb = nrb;
            }
        }
    }
    if (fabs(p) < pivtiny) p = (p < R(0)) ? -pivtiny : pivtiny;
    u0[(int64_t)(n - 1) * s] = p;
    R y2 = R(0), y1 = tdiv(rb, p);
    y[(int64_t)(n - 1) * s] = y1;
    for (int i0 = n - 2; i0 >= 0; i0 -= TRI_PF) {
        R f0[TRI_PF], f1[TRI_PF], f2[TRI_PF], fy[TRI_PF];
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 - u;
            const bool ok = i >= 0;
            f0[u] = ok ? u0[(int64_t)i * s] : R(1);
            f1[u] = ok ? u1[(int64_t)i * s] : R(0);
            f2[u] = ok ? u2[(int64_t)i * s] : R(0);
            fy[u] = ok ? y[(int64_t)i * s] : R(0);
        }
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 - u;
            if (i < 0) break;
            R up = f0[u];
            if (fabs(up) < pivtiny) up = (up < R(0)) ? -pivtiny : pivtiny;
            const R yi = tdiv(fy[u] - f1[u] * y1 - f2[u] * y2, up);
            y[(int64_t)i * s] = yi;
            y2 = y1;
            y1 = yi;
        }
    }
}



template <class In>
__device__ void tri_solve_packed(const In& in, int n, float lam, float pivtiny, float* y, float4* F, int64_t s) {
    float p = in.dv(0) - lam, q = (n > 1) ? in.ev(0) : 0.f, r = 0.f, rb = y[0];
    for (int i0 = 0; i0 < n - 1; i0 += TRI_PF) {
        // right-hand sides of the next TRI_PF rows, loaded before the dependent chain uses them
        float b1v[TRI_PF];
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) b1v[u] = (i0 + u < n - 1) ? y[(int64_t)(i0 + u + 1) * s] : 0.f;
        // keep the loads together ahead of the chain (the compiler would otherwise sink each one
        // to its use and expose its latency at every step)
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) asm volatile("" ::"f"(b1v[u]));
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 + u;
            if (i >= n - 1) break;
            const float a = in.ev(i);
            const float bb = in.dv(i + 1) - lam;
            const float cc = (i + 1 < n - 1) ? in.ev(i + 1) : 0.f;
            const float b1 = b1v[u];
            if (fabsf(a) <= fabsf(p)) {
                if (p == 0.f) p = pivtiny;
                const float l = tdiv(a, p);
                F[(int64_t)i * s] = make_float4(p, q, r, rb);
                p = bb - l * q; q = cc - l * r; r = 0.f; rb = b1 - l * rb;
            } else {
                const float l = tdiv(p, a);
                F[(int64_t)i * s] = make_float4(a, bb, cc, b1);
                const float np = q - l * bb, nq = r - l * cc, nrb = rb - l * b1;
                p = np; q = nq; r = 0.f; rb = nrb;
            }
        }
    }
    if (fabsf(p) < pivtiny) p = (p < 0.f) ? -pivtiny : pivtiny;
    float y2 = 0.f, y1 = tdiv(rb, p);
    y[(int64_t)(n - 1) * s] = y1;
    for (int i0 = n - 2; i0 >= 0; i0 -= TRI_PF) {
        float4 fv[TRI_PF];
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u)
            fv[u] = (i0 - u >= 0) ? F[(int64_t)(i0 - u) * s] : make_float4(1.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) asm volatile("" ::"f"(fv[u].x), "f"(fv[u].y), "f"(fv[u].z), "f"(fv[u].w));
#pragma unroll
        for (int u = 0; u < TRI_PF; ++u) {
            const int i = i0 - u;
            if (i < 0) break;
            const float4 f = fv[u];
            float up = f.x;
            if (fabsf(up) < pivtiny) up = (up < 0.f) ? -pivtiny : pivtiny;
            const float yi = tdiv(f.w - f.y * y1 - f.z * y2, up);
            y[(int64_t)i * s] = yi;
            y2 = y1;
            y1 = yi;
        }
    }
}

// Inverse iteration.  FP64: the iterate lives in Y itself and the factors in work (3 n^2
// doubles).  FP32: the packed factors (n^2 float4) and the iterate (n^2 floats) are at the start
// of work, and the normalised iterate is written to Y (FP64) at the end.
template <class R>
__global__ void __launch_bounds__(128) k_inviter(const MmfDesc* __restrict__ descs,
                                                 const int* __restrict__ idx,
                                                 const double* __restrict__ dvec,
                                                 const double* __restrict__ evec,
                                                 const double* __restrict__ aux,
                                                 const double* __restrict__ Eg,
                                                 double* __restrict__ Yg,
                                                 double* __restrict__ work, int iters) {
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const TriIn<R> in(d, dvec, evec, evec, aux + 8 * sid, (const float*)work);
    const double* E = Eg + d.vec_off;
    const double sc = in.scale;
    const double tnd = aux[8 * sid + 3] * sc;
    const double ortol = (double)TriP<R>::ortol * tnd;
    const R eps = TriP<R>::eps();
    const R tn = R(tnd);
    int kbeg = k, kend = k + 1;
    R lam_first = R(E[k] * sc);
    if constexpr (sizeof(R) == 4) {
        // FP32 (mixed path): every vector on its own; clusters are orthonormalised afterwards by
        // k_cluster_cgs2_f32.  Numerically equal eigenvalues (gaps below pert) get staggered shifts
        // so that their iterates differ: shift = lam of the first of the run + (position) pert.
        int k1 = k;
        while (k1 > 0) {
            const R a = R(E[k1 - 1] * sc), b = R(E[k1] * sc);
            if (b - a >= R(10) * eps * fmax(fabs(b), tn * R(1e-3))) break;
            --k1;
        }
        const R l1 = R(E[k1] * sc);
        lam_first = l1 + R(k - k1) * (R(10) * eps * fmax(fabs(l1), tn * R(1e-3)));
        if (lam_first < R(E[k] * sc)) lam_first = R(E[k] * sc);
    } else {
        if (k > 0 && (E[k] - E[k - 1]) * sc <= ortol) return;  // not the first of its cluster
        while (kend < n && (E[kend] - E[kend - 1]) * sc <= ortol) ++kend;
    }
    const R pivtiny = eps * fmax(tn, R(1e-30));
    const int64_t s = n;  // row stride of the row-major arrays
    const int64_t nn = (int64_t)n * n;
    R* base = sizeof(R) == 8 ? (R*)(work + 3 * d.sq_off) : (R*)tri_f32_base((const float*)work, d);
    R* u0 = base;
    R* u1 = u0 + nn;
    R* u2 = u1 + nn;
    float4* F = (float4*)base;  // FP32: packed factors (4 n^2 floats), then the iterate
    R* Yw = sizeof(R) == 8 ? (R*)(Yg + d.sq_off) : base + 4 * nn;
    R lamprev = R(0);
    for (int j = kbeg; j < kend; ++j) {
        R lam = (j == k) ? lam_first : R(E[j] * sc);
        if (j > k) {
            const R pert = R(10) * eps * fmax(fabs(lam), tn * R(1e-3));
            if (lam - lamprev < pert) lam = lamprev + pert;
        }
        lamprev = lam;
        R* y = Yw + j;
        R* a0 = u0 + j;
        R* a1 = u1 + j;
        R* a2 = u2 + j;
        for (int i = 0; i < n; ++i)
            y[(int64_t)i * s] = hash_unit<R>(((uint64_t)sid << 40) ^ ((uint64_t)j << 20) ^ (uint64_t)i);
        for (int it = 0; it < iters; ++it) {
            if constexpr (sizeof(R) == 4)
                tri_solve_packed(in, n, lam, pivtiny, (float*)y, F + j, s);
            else
                tri_solve<R>(in, n, lam, pivtiny, y, a0, a1, a2, s);
            // FP64: orthogonalise against the cluster's earlier vectors
            for (int jp = k; jp < j && sizeof(R) == 8; ++jp) {
                const R* z = Yw + jp;
                R dot = R(0);
#pragma unroll 8
                for (int i = 0; i < n; ++i) dot += y[(int64_t)i * s] * z[(int64_t)i * s];
#pragma unroll 8
                for (int i = 0; i < n; ++i) y[(int64_t)i * s] -= dot * z[(int64_t)i * s];
            }
            R mx = R(0);
#pragma unroll 8
            for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(y[(int64_t)i * s]));
            const R inv1 = (mx > R(0)) ? R(1) / mx : R(1);
            R nrm = R(0);
#pragma unroll 8
            for (int i = 0; i < n; ++i) {
                R v = y[(int64_t)i * s] * inv1;
                nrm += v * v;
            }
            const R inv = inv1 / sqrt(nrm);
#pragma unroll 8
            for (int i = 0; i < n; ++i) y[(int64_t)i * s] *= inv;
        }
    }
}

// FP32 clusters: eigenvalues closer than ortol ||T|| are orthonormalised by one CTA each
// (the refinement that follows resolves the eigenvectors inside the cluster).  The cluster's m
// columns of the row-major iterate are copied to contiguous columns of a scratch area (the
// inverse iteration's factors, free by now: columns k .. kend-1 of an n x n column-major array,
// so that clusters never overlap), orthonormalised there by classical Gram-Schmidt applied twice
// per column ("twice is enough", Giraud, Langou & Rozloznik 2005): all dot products with the
// earlier columns at once (one warp per column), then one update pass over the rows; and copied
// back.  Work O(m^2 n) per cluster with O(m) barriers, coalesced in both layouts.
#define CL_THREADS 256
__global__ void __launch_bounds__(CL_THREADS) k_cluster_cgs2_f32(const MmfDesc* __restrict__ descs,
                                                                 const int* __restrict__ idx,
                                                                 const double* __restrict__ aux,
                                                                 const double* __restrict__ Eg,
                                                                 double* __restrict__ work) {
    __shared__ float dots[TRI_CMAX];
    __shared__ float red[CL_THREADS / 32];
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const int k = blockIdx.x;
    if (k >= n) return;
    const double* E = Eg + d.vec_off;
    const double ortol = (double)TriP<float>::ortol * aux[8 * sid + 3];
    if (k > 0 && E[k] - E[k - 1] <= ortol) return;  // not the first of its cluster
    int kend = k + 1;
    while (kend < n && E[kend] - E[kend - 1] <= ortol) ++kend;
    const int m = kend - k;
    if (m < 2) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t nn = (int64_t)n * n;
    float* Yw = tri_f32_base((const float*)work, d) + 4 * nn;  // row-major iterate
    float* Sc = tri_f32_base((const float*)work, d);           // scratch, column-major
    // gather: Sc[(k + j) n + i] = Yw[i n + k + j]
    for (int64_t e = tid; e < (int64_t)m * n; e += CL_THREADS) {
        const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
        Sc[(int64_t)(k + j) * n + i] = Yw[(int64_t)i * n + k + j];
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        float* y = Sc + (int64_t)(k + j) * n;
        for (int pass = 0; pass < 2 && j > 0; ++pass) {
            // dots with the earlier columns (chunks of TRI_CMAX), then y -= sum dots z
            for (int j0 = 0; j0 < j; j0 += TRI_CMAX) {
                const int jn = min(TRI_CMAX, j - j0);
                for (int jp = warp; jp < jn; jp += CL_THREADS / 32) {
                    const float* z = Sc + (int64_t)(k + j0 + jp) * n;
                    float acc = 0.f;
                    for (int i = lane; i < n; i += 32) acc = fmaf(y[i], z[i], acc);
                    acc = warp_sum(acc);
                    if (lane == 0) dots[jp] = acc;
                }
                __syncthreads();
                for (int i = tid; i < n; i += CL_THREADS) {
                    float v = y[i];
                    for (int jp = 0; jp < jn; ++jp) v = fmaf(-dots[jp], Sc[(int64_t)(k + j0 + jp) * n + i], v);
                    y[i] = v;
                }
                __syncthreads();
            }
        }
        float part = 0.f;
        for (int i = tid; i < n; i += CL_THREADS) part = fmaf(y[i], y[i], part);
        part = warp_sum(part);
        if (lane == 0) red[warp] = part;
        __syncthreads();
        float nrm = 0.f;
#pragma unroll
        for (int w = 0; w < CL_THREADS / 32; ++w) nrm += red[w];
        const float inv = nrm > 0.f ? rsqrtf(nrm) : 0.f;
        for (int i = tid; i < n; i += CL_THREADS) y[i] *= inv;
        __syncthreads();
    }
    // scatter back
    for (int64_t e = tid; e < (int64_t)m * n; e += CL_THREADS) {
        const int i = (int)(e / m), j = (int)(e - (int64_t)i * m);
        Yw[(int64_t)i * n + k + j] = Sc[(int64_t)(k + j) * n + i];
    }
}

// Y (FP64, row-major) from the FP32 iterates
__global__ void __launch_bounds__(256) k_widen_y_f32(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                     const double* __restrict__ work, double* __restrict__ Yg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int64_t nn = (int64_t)d.n * d.n;
    const float* Yw = tri_f32_base((const float*)work, d) + 4 * nn;
    double* Y = Yg + d.sq_off;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x)
        Y[e] = (double)Yw[e];
}

cudaError_t mmf_launch_tridiag_eig(const MmfLaunch& L, const double* dvec, const double* evec,
                                   double* aux, double* e2, double* E, double* Y, double* work,
                                   int* status, int fp32, int iters) {
    if (L.count <= 0) return cudaSuccess;
    k_tri_prep<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, dvec, evec, aux, e2, fp32 ? (float*)work : nullptr);
    dim3 g((L.nmax + 127) / 128, L.count);
    if (fp32) {
        k_bisect<float><<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, e2, aux, (const float*)work, E, status);
        k_inviter<float><<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, evec, aux, E, Y, work, iters);
        k_cluster_cgs2_f32<<<dim3(L.nmax, L.count), CL_THREADS, 0, L.stream>>>(L.desc, L.idx, aux, E, work);
        k_widen_y_f32<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, work, Y);
    } else {
        k_bisect<double><<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, e2, aux, nullptr, E, status);
        k_inviter<double><<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, evec, aux, E, Y, work, iters);
    }
    return cudaGetLastError();
}
