// k_tridiag.cu -- S4: eigenpairs of the real symmetric tridiagonal T = tridiag(e, d, e), FP64.
//
// Eigenvalues by Sturm-sequence bisection (Givens 1954; Barth, Martin & Wilkinson 1967):
// count(x) = number of sign changes of the leading principal minors of T - x I (a division-
// free three-term recurrence).  One thread per eigenvalue, each bracketing its own index
// inside the Gershgorin interval until the bracket is below max(2 eps max(|lo|,|hi|), tol |T|)
// (tol = eps for the FP64 path; 1e-10 when the refinement follows, as T is then FP32-accurate).
//
// Eigenvectors by inverse iteration (Wilkinson 1965): (T - lambda I) y = b solved by
// Gaussian elimination with partial pivoting on the tridiagonal band, a fixed number of
// iterations (3) from a hashed start vector.  Eigenvalues closer than ortol = 1e-4 ||T||_1 form a cluster; one
// thread handles a whole cluster in ascending order and orthogonalises each iterate against
// the cluster's earlier vectors (modified Gram-Schmidt), as LAPACK's stein does.
// Y is written row-major: Y[i * n + k] = component i of eigenvector k.
#include "mmf_internal.h"

#define TRI_ORTOL 1e-4

__device__ __forceinline__ double dmax(double a, double b) { return a > b ? a : b; }

// per system: gl, gu, pivmin, tnorm
__global__ void k_tri_prep(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                           const double* __restrict__ dvec, const double* __restrict__ evec,
                           double* __restrict__ aux, double* __restrict__ e2vec) {
    __shared__ double red[4][32];
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
    }
}

// Sturm count by the three-term recurrence of the leading principal minors,
//   p_0 = 1, p_1 = d_0 - x, p_{i+1} = (d_i - x) p_i - e_{i-1}^2 p_{i-1},
// counting sign changes (= eigenvalues below x); an exact zero takes the sign opposite to its
// predecessor (a negative pivot, as in the ratio form).  Every 16 steps the pair (p_i, p_{i-1})
// is rescaled by the power of two that brings the larger of the two below 1, which changes no
// sign and keeps 16 further steps far from overflow.
__device__ __forceinline__ int sturm_count(const double* __restrict__ dd,
                                           const double* __restrict__ e2, int n, double x) {
    int cnt = 0;
    double pm = 1.0, p = dd[0] - x;
    if (p == 0.0) p = -1e-300;
    cnt += (p < 0.0);
    for (int i = 1; i < n; ++i) {
        double pn = fma(dd[i] - x, p, -e2[i - 1] * pm);
        if (pn == 0.0) pn = (p < 0.0) ? 1e-300 : -1e-300;
        cnt += ((pn < 0.0) != (p < 0.0));
        pm = p;
        p = pn;
        if ((i & 15) == 0) {
            int ex;
            frexp(fmax(fabs(p), fabs(pm)), &ex);
            const double sc = ldexp(1.0, -ex);
            p *= sc;
            pm *= sc;
        }
    }
    return cnt;
}

__global__ void __launch_bounds__(128) k_bisect(const MmfDesc* __restrict__ descs,
                                                const int* __restrict__ idx,
                                                const double* __restrict__ dvec,
                                                const double* __restrict__ e2vec,
                                                const double* __restrict__ aux,
                                                double* __restrict__ Eout,
                                                int* __restrict__ status, double rel_tol) {
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* dd = dvec + d.vec_off;
    const double* e2 = e2vec + d.vec_off;
    double lo = aux[8 * sid], hi = aux[8 * sid + 1];
    const double pivmin = aux[8 * sid + 2];
    const double tn = aux[8 * sid + 3];
    const double eps = 2.220446049250313e-16;
    int it = 0;
    for (; it < 200; ++it) {
        double tol = dmax(2.0 * eps * dmax(fabs(lo), fabs(hi)), rel_tol * tn) + pivmin;
        if (hi - lo <= tol) break;
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (sturm_count(dd, e2, n, mid) <= k) lo = mid;
        else hi = mid;
    }
    Eout[d.vec_off + k] = 0.5 * (lo + hi);
    if (it >= 200) status[sid] = MMF_ST_NOCONV;
}

__device__ __forceinline__ double hash_unit(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Solve (T - lam I) y = y in place; u0/u1/u2 are the (strided) U factor arrays.
__device__ void tri_solve(const double* __restrict__ dd, const double* __restrict__ ee, int n,
                          double lam, double pivtiny, double* y, double* u0, double* u1,
                          double* u2, int64_t s) {
    double p = dd[0] - lam, q = (n > 1) ? ee[0] : 0.0, r = 0.0, rb = y[0];
    for (int i = 0; i < n - 1; ++i) {
        const double a = ee[i];
        const double bb = dd[i + 1] - lam;
        const double cc = (i + 1 < n - 1) ? ee[i + 1] : 0.0;
        const double b1 = y[(int64_t)(i + 1) * s];
        if (fabs(a) <= fabs(p)) {
            if (p == 0.0) p = pivtiny;
            const double l = a / p;
            u0[(int64_t)i * s] = p; u1[(int64_t)i * s] = q; u2[(int64_t)i * s] = r;
            y[(int64_t)i * s] = rb;
            p = bb - l * q; q = cc - l * r; r = 0.0; rb = b1 - l * rb;
        } else {
            const double l = p / a;
            u0[(int64_t)i * s] = a; u1[(int64_t)i * s] = bb; u2[(int64_t)i * s] = cc;
            y[(int64_t)i * s] = b1;
            const double np = q - l * bb, nq = r - l * cc, nrb = rb - l * b1;
            p = np; q = nq; r = 0.0; rb = nrb;
        }
    }
    if (fabs(p) < pivtiny) p = (p < 0.0) ? -pivtiny : pivtiny;
    u0[(int64_t)(n - 1) * s] = p;
    // back substitution
    double y2 = 0.0, y1 = rb / p;
    y[(int64_t)(n - 1) * s] = y1;
    for (int i = n - 2; i >= 0; --i) {
        double up = u0[(int64_t)i * s];
        if (fabs(up) < pivtiny) up = (up < 0.0) ? -pivtiny : pivtiny;
        const double yi = (y[(int64_t)i * s] - u1[(int64_t)i * s] * y1 - u2[(int64_t)i * s] * y2) / up;
        y[(int64_t)i * s] = yi;
        y2 = y1;
        y1 = yi;
    }
}

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
    const double* dd = dvec + d.vec_off;
    const double* ee = evec + d.vec_off;
    const double* E = Eg + d.vec_off;
    const double tn = aux[8 * sid + 3];
    const double ortol = TRI_ORTOL * tn;
    if (k > 0 && E[k] - E[k - 1] <= ortol) return;  // not the first of its cluster
    int kend = k + 1;
    while (kend < n && E[kend] - E[kend - 1] <= ortol) ++kend;
    const double eps = 2.220446049250313e-16;
    const double pivtiny = eps * fmax(tn, 1e-300);
    const int64_t s = n;  // row stride of the row-major arrays
    double* Y = Yg + d.sq_off;
    double* u0 = work + 3 * d.sq_off;
    double* u1 = u0 + (int64_t)n * n;
    double* u2 = u1 + (int64_t)n * n;
    double lamprev = 0.0;
    for (int j = k; j < kend; ++j) {
        double lam = E[j];
        if (j > k) {
            const double pert = 10.0 * eps * fmax(fabs(lam), tn * 1e-3);
            if (lam - lamprev < pert) lam = lamprev + pert;
        }
        lamprev = lam;
        double* y = Y + j;
        double* a0 = u0 + j;
        double* a1 = u1 + j;
        double* a2 = u2 + j;
        for (int i = 0; i < n; ++i) y[(int64_t)i * s] = hash_unit(((uint64_t)sid << 40) ^ ((uint64_t)j << 20) ^ (uint64_t)i);
        for (int it = 0; it < iters; ++it) {
            tri_solve(dd, ee, n, lam, pivtiny, y, a0, a1, a2, s);
            // orthogonalise against the cluster's earlier vectors
            for (int jp = k; jp < j; ++jp) {
                const double* z = Y + jp;
                double dot = 0.0;
                for (int i = 0; i < n; ++i) dot += y[(int64_t)i * s] * z[(int64_t)i * s];
                for (int i = 0; i < n; ++i) y[(int64_t)i * s] -= dot * z[(int64_t)i * s];
            }
            double mx = 0.0;
            for (int i = 0; i < n; ++i) mx = fmax(mx, fabs(y[(int64_t)i * s]));
            const double inv1 = (mx > 0.0) ? 1.0 / mx : 1.0;
            double nrm = 0.0;
            for (int i = 0; i < n; ++i) {
                double v = y[(int64_t)i * s] * inv1;
                nrm += v * v;
            }
            const double inv = inv1 / sqrt(nrm);
            for (int i = 0; i < n; ++i) y[(int64_t)i * s] *= inv;
        }
    }
}

cudaError_t mmf_launch_tridiag_eig(const MmfLaunch& L, const double* dvec, const double* evec,
                                   double* aux, double* e2, double* E, double* Y, double* work,
                                   int* status, double rel_tol, int iters) {
    if (L.count <= 0) return cudaSuccess;
    k_tri_prep<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, dvec, evec, aux, e2);
    dim3 g((L.nmax + 127) / 128, L.count);
    k_bisect<<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, e2, aux, E, status, rel_tol);
    k_inviter<<<g, 128, 0, L.stream>>>(L.desc, L.idx, dvec, evec, aux, E, Y, work, iters);
    return cudaGetLastError();
}
