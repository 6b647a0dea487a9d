// k_refine.cu -- S6: Ogita-Aishima refinement of approximate eigenpairs (mixed path).
//
// Ogita & Aishima, "Iterative refinement for symmetric eigenvalue decomposition",
// Japan J. Indust. Appl. Math. 35 (2018), complexified.  For approximate eigenvectors X of
// the Hermitian H_F (columns, near orthonormal):
//     G = X^H X (r_ij = delta_ij - g_ij),  S = X^H H_F X,
//     lam_i = s_ii / g_ii,
//     Et_ij = (s_ij - lam_j g_ij) / (lam_j - lam_i)   for well separated pairs,
//     Et_ij = r_ij / 2                                 on the diagonal and inside clusters,
//     X <- X + X Et.
// Products that decide the result (G, S) are formed FP64-accurately from FP32 pieces: every
// FP64 value is split x = x1 + x2 (x1 = fl32(x), x2 = fl32(x - x1)); x1*y1 is taken exactly
// (product + FMA error term), the cross terms in FP32, and the sums are accumulated in
// double-FP32 (TwoSum, Knuth 1969).  X Et only needs FP32 (Et is small).  H_F X is applied in
// FP64 from the coefficients, never from the FP32 matrix.
// A pair is treated as clustered when |lam_i - lam_j| <= 20 |s_ij - lam_j g_ij| (the first-order
// correction would exceed 0.05) or the gap is below 1e-13 |H_F|; consecutive clustered indices
// form a cluster whose eigenvectors are separated by an FP64 Jacobi solve of the small
// projected matrix X_C^H H_F X_C (clusters of up to RF_CMAX vectors).
#include "mmf_internal.h"

#define RF_TILE 32
#define RF_KC 32
#define RF_KG 16   // k-chunk of the FP64-accurate Gram kernel
#define RF_CMAX 32
#define RF_TAU 20.0

// ------------------------------------------------------------------ HX = H_F X (FP64, sparse)
__global__ void __launch_bounds__(256) k_apply_hf(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx,
                                                  const double2* __restrict__ coef,
                                                  const double2* __restrict__ Xg,
                                                  double2* __restrict__ HXg, int col0, int ncols) {
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, D = d.D;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int cbeg = col0 + blockIdx.y * 16;
    if (r >= n || cbeg >= n) return;
    const int cend = min(min(cbeg + 16, n), col0 + ncols);
    const int b = r / D, i = r - b * D;
    int nv[MMF_MAX_MODES];
    block_nvec(d, b, nv);
    const double sh = block_ndotw(d, b);
    const double2* H0 = coef + d.coef_off;
    const double2* X = Xg + d.mat_off;
    double2* HX = HXg + d.mat_off;
    for (int c = cbeg; c < cend; ++c) {
        const double2* x = X + (int64_t)c * d.ld;
        double2 acc = make_double2(0.0, 0.0);
        for (int j = 0; j < D; ++j) acc = acc + H0[i * D + j] * x[j + D * b];
        acc = acc - sh * x[r];
        int64_t off = d.coef_off + (int64_t)D * D;
        for (int l = 0; l < d.K; ++l) {
            for (int h = 1; h <= d.nharm[l]; ++h) {
                const double2* V = coef + off + (int64_t)(h - 1) * D * D;
                if (nv[l] + h <= d.N[l]) {
                    const int bu = b + h * d.S[l];
                    for (int j = 0; j < D; ++j) acc = acc + V[i * D + j] * x[j + D * bu];
                }
                if (nv[l] - h >= -d.N[l]) {
                    const int bd = b - h * d.S[l];
                    for (int j = 0; j < D; ++j) acc = acc + cmulc(V[j * D + i], x[j + D * bd]);
                }
            }
            off += (int64_t)d.nharm[l] * D * D;
        }
        HX[(int64_t)c * d.ld + r] = acc;
    }
}

// ------------------------------------------------------------------ G = X^H X, S = X^H HX
// Upper-triangle tiles (I <= J) of 32 x 32; both triangles are written.  X1 = true: X holds
// FP32-exact values (the first refinement step), so its second pieces vanish and are skipped.
template <bool X1>
__device__ __forceinline__ void gram_cmacc(DF& gre, DF& gim, DF& sre, DF& sim, const Split& a,
                                           const Split& b, const Split& h) {
    if (X1) {
        // conj(a) b with a, b FP32-exact; conj(a) h with h split
        df_mac11(gre, a.r1, b.r1);
        df_mac11(gre, a.i1, b.i1);
        df_mac11(gim, a.r1, b.i1);
        df_mac11(gim, -a.i1, b.r1);
        df_mac1(sre, a.r1, h.r1, h.r2);
        df_mac1(sre, a.i1, h.i1, h.i2);
        df_mac1(sim, a.r1, h.i1, h.i2);
        df_mac1(sim, -a.i1, h.r1, h.r2);
    } else {
        df_cmacc(gre, gim, a, b);
        df_cmacc(sre, sim, a, h);
    }
}

template <bool X1>
__global__ void __launch_bounds__(256) k_gram_df32(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Xg,
                                                   const double2* __restrict__ HXg,
                                                   double2* __restrict__ Gg,
                                                   double2* __restrict__ Sg) {
    __shared__ Split xi[RF_KG][RF_TILE + 1];
    __shared__ Split xj[RF_KG][RF_TILE + 1];
    __shared__ Split hj[RF_KG][RF_TILE + 1];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int T = (n + RF_TILE - 1) / RF_TILE;
    // tile index -> (I, J), I <= J
    int t = blockIdx.x, I = 0;
    if (t >= T * (T + 1) / 2) return;
    while (t >= T - I) { t -= T - I; ++I; }
    const int J = I + t;
    const int i0 = I * RF_TILE, j0 = J * RF_TILE;
    const double2* X = Xg + d.mat_off;
    const double2* HX = HXg + d.mat_off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // outputs (ty + 16a, tx + 16b)
    DF gr[2][2], gi[2][2], sr[2][2], si[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            gr[a][b] = gi[a][b] = sr[a][b] = si[a][b] = DF{0.f, 0.f};
        }
    for (int k0 = 0; k0 < n; k0 += RF_KG) {
        for (int e = threadIdx.x; e < RF_KG * RF_TILE; e += 256) {
            const int c = e / RF_KG, kk = e - c * RF_KG;
            const int k = k0 + kk;
            const double2 z = make_double2(0.0, 0.0);
            xi[kk][c] = split((k < n && i0 + c < n) ? X[(int64_t)(i0 + c) * d.ld + k] : z);
            xj[kk][c] = split((k < n && j0 + c < n) ? X[(int64_t)(j0 + c) * d.ld + k] : z);
            hj[kk][c] = split((k < n && j0 + c < n) ? HX[(int64_t)(j0 + c) * d.ld + k] : z);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RF_KG; ++kk) {
            const Split a0 = xi[kk][ty], a1 = xi[kk][ty + 16];
            const Split b0 = xj[kk][tx], b1 = xj[kk][tx + 16];
            const Split h0 = hj[kk][tx], h1 = hj[kk][tx + 16];
            gram_cmacc<X1>(gr[0][0], gi[0][0], sr[0][0], si[0][0], a0, b0, h0);
            gram_cmacc<X1>(gr[0][1], gi[0][1], sr[0][1], si[0][1], a0, b1, h1);
            gram_cmacc<X1>(gr[1][0], gi[1][0], sr[1][0], si[1][0], a1, b0, h0);
            gram_cmacc<X1>(gr[1][1], gi[1][1], sr[1][1], si[1][1], a1, b1, h1);
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                df_renorm(gr[a][b]); df_renorm(gi[a][b]); df_renorm(sr[a][b]); df_renorm(si[a][b]);
            }
        __syncthreads();
    }
    double2* G = Gg + d.mat_off;
    double2* S = Sg + d.mat_off;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < n && j < n && (I < J || i <= j)) {
                double2 g = df_value(gr[a][b], gi[a][b]);
                double2 s = df_value(sr[a][b], si[a][b]);
                if (i == j) { g.y = 0.0; s.y = 0.0; }
                G[(int64_t)j * d.ld + i] = g;
                S[(int64_t)j * d.ld + i] = s;
                G[(int64_t)i * d.ld + j] = conj(g);
                S[(int64_t)i * d.ld + j] = conj(s);
            }
        }
}

// ------------------------------------------------------------------ lam, clusters
// One CTA per system: lam_i = s_ii / g_ii; link_i = pair (i, i+1) clustered; cluster id = the
// first index of its run.  aux per system: cid (n ints) stored in the E2 buffer's tail.
__global__ void __launch_bounds__(256) k_oa_lambda(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Gg,
                                                   const double2* __restrict__ Sg,
                                                   double* __restrict__ lamg,
                                                   int* __restrict__ cidg) {
    const MmfDesc d = descs[idx[blockIdx.x]];
    const int n = d.n;
    const double2* G = Gg + d.mat_off;
    const double2* S = Sg + d.mat_off;
    double* lam = lamg + d.vec_off;
    int* cid = cidg + d.vec_off;
    __shared__ double hmax;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        lam[i] = S[(int64_t)i * d.ld + i].x / G[(int64_t)i * d.ld + i].x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(lam[i]));
        hmax = m;
    }
    __syncthreads();
    // link flags into cid (1 = linked to the next)
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int link = 0;
        if (i + 1 < n) {
            const double gap = fabs(lam[i + 1] - lam[i]);
            const double2 s = S[(int64_t)(i + 1) * d.ld + i], g = G[(int64_t)(i + 1) * d.ld + i];
            const double2 num = s - lam[i + 1] * g;
            link = (gap <= RF_TAU * sqrt(abs2(num))) || (gap <= 1e-13 * hmax);
        }
        cid[i] = link;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int start = 0, prev = 0;
        for (int i = 0; i < n; ++i) {
            const int link = cid[i];
            if (i == 0 || !prev) start = i;
            cid[i] = start;
            prev = link;
        }
    }
}

// Et in place of G (diagonal and clustered pairs: r/2; others: OA formula)
__global__ void __launch_bounds__(256) k_oa_etilde(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   double2* __restrict__ Gg,
                                                   const double2* __restrict__ Sg,
                                                   const double* __restrict__ lamg,
                                                   const int* __restrict__ cidg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int64_t tot = (int64_t)n * n;
    double2* G = Gg + d.mat_off;
    const double2* S = Sg + d.mat_off;
    const double* lam = lamg + d.vec_off;
    const int* cid = cidg + d.vec_off;
    double hmax = fmax(fabs(lam[0]), fabs(lam[n - 1]));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
        const int64_t o = (int64_t)j * d.ld + i;
        const double2 g = G[o];
        double2 et;
        if (i == j) {
            et = make_double2(0.5 * (1.0 - g.x), 0.0);
        } else {
            const double2 num = S[o] - lam[j] * g;
            const double gap = lam[j] - lam[i];
            const bool clustered = cid[i] == cid[j] || fabs(gap) <= RF_TAU * sqrt(abs2(num)) ||
                                   fabs(gap) <= 1e-13 * fmax(hmax, fabs(lam[i]));
            et = clustered ? (-0.5) * g : (1.0 / gap) * num;
        }
        G[o] = et;
    }
}

// ------------------------------------------------------------------ Xn = X + X Et (FP32 GEMM)
__global__ void __launch_bounds__(256) k_xe_update(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Xg,
                                                   const double2* __restrict__ Etg,
                                                   double2* __restrict__ Xn) {
    __shared__ float2 xs[RF_KC][64 + 1];
    __shared__ float2 es[RF_KC][64 + 1];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n;
    const int r0 = blockIdx.x * 64, c0 = blockIdx.y * 64;
    if (r0 >= n || c0 >= n) return;
    const double2* X = Xg + d.mat_off;
    const double2* Et = Etg + d.mat_off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // rows tx + 16a, cols ty + 16b
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
    for (int k0 = 0; k0 < n; k0 += RF_KC) {
        for (int e = threadIdx.x; e < RF_KC * 64; e += 256) {
            // X tile: rows r0..r0+63, cols k0..k0+31 (coalesced over rows)
            const int kk = e / 64, rr = e - kk * 64;
            const int r = r0 + rr, k = k0 + kk;
            double2 v = (r < n && k < n) ? X[(int64_t)k * d.ld + r] : make_double2(0.0, 0.0);
            xs[kk][rr] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
            // Et tile: rows k0..k0+31, cols c0..c0+63 (coalesced over k)
            const int cc = e / RF_KC, k2 = e - cc * RF_KC;
            const int c = c0 + cc, kr = k0 + k2;
            double2 w = (c < n && kr < n) ? Et[(int64_t)c * d.ld + kr] : make_double2(0.0, 0.0);
            es[k2][cc] = make_float2(__double2float_rn(w.x), __double2float_rn(w.y));
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RF_KC; ++kk) {
            float2 xa[4], eb[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) xa[a] = xs[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) eb[b] = es[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fmaf(xa[a].x, eb[b].x, fmaf(-xa[a].y, eb[b].y, acc[a][b].x));
                    acc[a][b].y = fmaf(xa[a].x, eb[b].y, fmaf(xa[a].y, eb[b].x, acc[a][b].y));
                }
        }
        __syncthreads();
    }
    double2* O = Xn + d.mat_off;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int r = r0 + tx + 16 * a, c = c0 + ty + 16 * b;
            if (r < n && c < n) {
                const int64_t o = (int64_t)c * d.ld + r;
                const double2 x = X[o];
                O[o] = make_double2(x.x + (double)acc[a][b].x, x.y + (double)acc[a][b].y);
            }
        }
}

// ------------------------------------------------------------------ Xn = X + X Et on tensor cores
// The complex product is a real product of twice the size,
//   [Re Y | Im Y] = [Re X, Im X] [[Re E, Im E], [-Im E, Re E]],
// taken on the tcgen05 engine in split TF32 (x = x1 + x2, x1 = tf32(x), x2 = tf32(x - x1);
// x y ~ x1 y1 + x1 y2 + x2 y1, about FP32 accuracy; Et is small, so that is ample).  Operands are
// K-major rows of la = round_up(2n, 4) floats, placed in buffers free at this point:
// B1 -> S, B2 -> HX (2n rows), A1 -> Zp (n rows), A2 and then C (n x 2n) -> the Et buffer after
// B has been built from it.
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ int xe_la(int n) { return (2 * n + 3) & ~3; }

__global__ void __launch_bounds__(256) k_xe_prep_B(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Etg,
                                                   double2* __restrict__ B1g, double2* __restrict__ B2g) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = xe_la(n);
    const double2* Et = Etg + d.mat_off;
    float* B1 = reinterpret_cast<float*>(B1g + d.mat_off);
    float* B2 = reinterpret_cast<float*>(B2g + d.mat_off);
    const int64_t tot = (int64_t)2 * n * la;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / la), k = (int)(e - (int64_t)j * la);
        float v = 0.f;
        if (k < 2 * n) {
            const int jj = j < n ? j : j - n, kk = k < n ? k : k - n;
            const double2 x = Et[(int64_t)jj * d.ld + kk];
            double w;
            if (j < n) w = (k < n) ? x.x : -x.y;
            else w = (k < n) ? x.y : x.x;
            v = (float)w;
        }
        const float v1 = tf32_round(v);
        B1[e] = v1;
        B2[e] = tf32_round(v - v1);
    }
}

__global__ void __launch_bounds__(256) k_xe_prep_A(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Xg,
                                                   float2* __restrict__ A1g, double2* __restrict__ A2g) {
    __shared__ double2 t[32][33];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, la = xe_la(n);
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    if (r0 >= n || c0 >= n) return;
    const double2* X = Xg + d.mat_off;
    float* A1 = reinterpret_cast<float*>(A1g + d.mat_off);
    float* A2 = reinterpret_cast<float*>(A2g + d.mat_off);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {  // X(r0 + tx, c0 + q), rows fastest
        const int r = r0 + tx, c = c0 + q;
        t[q][tx] = (r < n && c < n) ? X[(int64_t)c * d.ld + r] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {  // A[r0 + q][c0 + tx] (re) and A[r0 + q][n + c0 + tx] (im)
        const int r = r0 + q, c = c0 + tx;
        if (r < n && c < n) {
            const double2 x = t[tx][q];
            const float re = (float)x.x, im = (float)x.y;
            const float re1 = tf32_round(re), im1 = tf32_round(im);
            A1[(int64_t)r * la + c] = re1;
            A2[(int64_t)r * la + c] = tf32_round(re - re1);
            A1[(int64_t)r * la + n + c] = im1;
            A2[(int64_t)r * la + n + c] = tf32_round(im - im1);
        }
        if (r < n && c0 + 32 >= n && tx < la - 2 * n) {  // zero the row padding
            A1[(int64_t)r * la + 2 * n + tx] = 0.f;
            A2[(int64_t)r * la + 2 * n + tx] = 0.f;
        }
    }
}

__global__ void k_xe_jobs(const MmfDesc* __restrict__ descs, const int* __restrict__ idx, int count,
                          float2* Zp, double2* R, double2* S, double2* HX, UmmaJob* jobs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const MmfDesc d = descs[idx[i]];
    const int n = d.n, la = xe_la(n);
    const float* A1 = reinterpret_cast<const float*>(Zp + d.mat_off);
    const float* A2 = reinterpret_cast<const float*>(R + d.mat_off);
    const float* B1 = reinterpret_cast<const float*>(S + d.mat_off);
    const float* B2 = reinterpret_cast<const float*>(HX + d.mat_off);
    UmmaJob j;
    j.A[0] = A1; j.B[0] = B1;
    j.A[1] = A1; j.B[1] = B2;
    j.A[2] = A2; j.B[2] = B1;
    j.C = reinterpret_cast<float*>(R + d.mat_off) + (int64_t)n * la;
    j.M = n; j.N = 2 * n; j.K = 2 * n;
    j.lda = la; j.ldb = la; j.ldc = 2 * n;
    jobs[i] = j;
}

__global__ void __launch_bounds__(256) k_xe_apply(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx, double2* __restrict__ Xg,
                                                  const double2* __restrict__ R) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, la = xe_la(n);
    const float* C = reinterpret_cast<const float*>(R + d.mat_off) + (int64_t)n * la;
    double2* X = Xg + d.mat_off;
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), r = (int)(e - (int64_t)j * n);  // X(r, j), rows fastest
        const double2 x = X[(int64_t)j * d.ld + r];
        const float yr = C[(int64_t)r * 2 * n + j], yi = C[(int64_t)r * 2 * n + n + j];
        X[(int64_t)j * d.ld + r] = make_double2(x.x + (double)yr, x.y + (double)yi);
    }
}

// ------------------------------------------------------------------ cluster separation
// One CTA per system; clusters handled one after another.  For cluster C (m vectors):
// B = X_C^H H_F X_C in FP64 (H_F X_C from the HX buffer, recomputed for the new X), cyclic
// Jacobi on B, X_C <- X_C W, lam_C <- eigenvalues of B ascending.
// CTA-parallel two-sided Jacobi on the m x m Hermitian B (column-major, ld RF_CMAX), with the
// round-robin pivot order: each round rotates m/2 disjoint pairs at once.  W accumulates the
// rotations; w receives the eigenvalues (unsorted).  All threads of the CTA call it.
__device__ void cta_jacobi(double2* B, double2* W, int m, double* w, double* rot, int* pq, int* flag) {
    const int tid = threadIdx.x, T = blockDim.x;
    const int mm = (m + 1) & ~1;
    for (int e = tid; e < m * m; e += T) {
        const int i = e % m, j = e / m;
        W[i + j * RF_CMAX] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    }
    __syncthreads();
    double fro = 0.0;
    for (int e = 0; e < m * m; ++e) fro += abs2(B[(e % m) + (e / m) * RF_CMAX]);
    const double thr = 2.220446049250313e-16 * sqrt(fro);
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) *flag = 0;
        __syncthreads();
        for (int round = 0; round < mm - 1; ++round) {
            for (int k = tid; k < mm / 2; k += T) {
                const int a0 = (k == 0) ? 0 : ((k - 1 + round) % (mm - 1)) + 1;
                const int b0 = ((mm - 1 - k - 1 + round) % (mm - 1)) + 1;
                const int p = a0 < b0 ? a0 : b0, q = a0 < b0 ? b0 : a0;
                pq[2 * k] = p;
                pq[2 * k + 1] = q;
                double c = 1.0, sn = 0.0, cf = 1.0, sf = 0.0;
                if (q < m) {
                    const double2 apq = B[p + q * RF_CMAX];
                    const double r = sqrt(abs2(apq));
                    if (r > thr) {
                        const double app = B[p + p * RF_CMAX].x, aqq = B[q + q * RF_CMAX].x;
                        cf = apq.x / r;
                        sf = apq.y / r;
                        const double th = (aqq - app) / (2.0 * r);
                        const double t = (th >= 0.0 ? 1.0 : -1.0) / (fabs(th) + sqrt(1.0 + th * th));
                        c = 1.0 / sqrt(1.0 + t * t);
                        sn = t * c;
                        *flag = 1;
                    }
                }
                rot[4 * k] = c; rot[4 * k + 1] = sn; rot[4 * k + 2] = cf; rot[4 * k + 3] = sf;
            }
            __syncthreads();
            for (int e = tid; e < (mm / 2) * m; e += T) {  // columns of B and W
                const int k = e / m, r = e - k * m;
                const int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= m || rot[4 * k + 1] == 0.0) continue;
                const double c = rot[4 * k], sn = rot[4 * k + 1];
                const double2 em = make_double2(rot[4 * k + 2], -rot[4 * k + 3]);
                const double2 bp = B[r + p * RF_CMAX], bq = B[r + q * RF_CMAX] * em;
                B[r + p * RF_CMAX] = c * bp - sn * bq;
                B[r + q * RF_CMAX] = sn * bp + c * bq;
                const double2 wp = W[r + p * RF_CMAX], wq = W[r + q * RF_CMAX] * em;
                W[r + p * RF_CMAX] = c * wp - sn * wq;
                W[r + q * RF_CMAX] = sn * wp + c * wq;
            }
            __syncthreads();
            for (int e = tid; e < (mm / 2) * m; e += T) {  // rows of B
                const int k = e / m, col = e - k * m;
                const int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= m || rot[4 * k + 1] == 0.0) continue;
                const double c = rot[4 * k], sn = rot[4 * k + 1];
                const double2 ep = make_double2(rot[4 * k + 2], rot[4 * k + 3]);
                const double2 bp = B[p + col * RF_CMAX], bq = ep * B[q + col * RF_CMAX];
                B[p + col * RF_CMAX] = c * bp - sn * bq;
                B[q + col * RF_CMAX] = sn * bp + c * bq;
            }
            __syncthreads();
            for (int k = tid; k < mm / 2; k += T) {
                const int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= m || rot[4 * k + 1] == 0.0) continue;
                B[p + q * RF_CMAX] = B[q + p * RF_CMAX] = make_double2(0.0, 0.0);
                B[p + p * RF_CMAX].y = 0.0;
                B[q + q * RF_CMAX].y = 0.0;
            }
            __syncthreads();
        }
        const int any = *flag;
        __syncthreads();
        if (!any) break;
    }
    for (int i = tid; i < m; i += T) w[i] = B[i + i * RF_CMAX].x;
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_cluster_sep(const MmfDesc* __restrict__ descs,
                                                     const int* __restrict__ idx,
                                                     const double2* __restrict__ coef,
                                                     double2* __restrict__ Xg,
                                                     double2* __restrict__ HXg,
                                                     double* __restrict__ lamg,
                                                     const int* __restrict__ cidg,
                                                     int* __restrict__ status) {
    __shared__ double2 B[RF_CMAX * RF_CMAX];
    __shared__ double2 W[RF_CMAX * RF_CMAX];
    __shared__ double w[RF_CMAX];
    __shared__ int perm[RF_CMAX];
    __shared__ double rot[4 * (RF_CMAX / 2)];
    __shared__ int pq[RF_CMAX + 2];
    __shared__ int flag;
    const int sid = idx[blockIdx.x];
    const MmfDesc d = descs[sid];
    const int n = d.n, D = d.D;
    double2* X = Xg + d.mat_off;
    double2* HX = HXg + d.mat_off;
    double* lam = lamg + d.vec_off;
    const int* cid = cidg + d.vec_off;
    const double2* H0 = coef + d.coef_off;
    int c0 = 0;
    while (c0 < n) {
        int c1 = c0 + 1;
        while (c1 < n && cid[c1] == c0) ++c1;
        const int m = c1 - c0;
        if (m >= 2 && m <= RF_CMAX) {
            // HX_C = H_F X_C (FP64)
            for (int e = threadIdx.x; e < n * m; e += blockDim.x) {
                const int cc = e / n, r = e - cc * n;
                const int c = c0 + cc;
                const int b = r / D, i = r - b * D;
                int nv[MMF_MAX_MODES];
                block_nvec(d, b, nv);
                const double2* x = X + (int64_t)c * d.ld;
                double2 acc = make_double2(0.0, 0.0);
                for (int j = 0; j < D; ++j) acc = acc + H0[i * D + j] * x[j + D * b];
                acc = acc - block_ndotw(d, b) * x[r];
                int64_t off = d.coef_off + (int64_t)D * D;
                for (int l = 0; l < d.K; ++l) {
                    for (int h = 1; h <= d.nharm[l]; ++h) {
                        const double2* V = coef + off + (int64_t)(h - 1) * D * D;
                        if (nv[l] + h <= d.N[l])
                            for (int j = 0; j < D; ++j) acc = acc + V[i * D + j] * x[j + D * (b + h * d.S[l])];
                        if (nv[l] - h >= -d.N[l])
                            for (int j = 0; j < D; ++j) acc = acc + cmulc(V[j * D + i], x[j + D * (b - h * d.S[l])]);
                    }
                    off += (int64_t)d.nharm[l] * D * D;
                }
                HX[(int64_t)c * d.ld + r] = acc;
            }
            __syncthreads();
            // B = X_C^H HX_C, one warp per entry
            for (int e = threadIdx.x >> 5; e < m * m; e += blockDim.x >> 5) {
                const int p = e % m, q = e / m;
                const double2* xp = X + (int64_t)(c0 + p) * d.ld;
                const double2* hq = HX + (int64_t)(c0 + q) * d.ld;
                double2 acc = make_double2(0.0, 0.0);
                for (int r = threadIdx.x & 31; r < n; r += 32) acc = acc + cmulc(xp[r], hq[r]);
                acc.x = warp_sum(acc.x);
                acc.y = warp_sum(acc.y);
                if ((threadIdx.x & 31) == 0) B[p + q * RF_CMAX] = acc;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int p = 0; p < m; ++p)  // Hermitian part
                    for (int q = p; q < m; ++q) {
                        double2 a = B[p + q * RF_CMAX], b = B[q + p * RF_CMAX];
                        double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
                        B[p + q * RF_CMAX] = h;
                        B[q + p * RF_CMAX] = conj(h);
                        if (p == q) B[p + p * RF_CMAX].y = 0.0;
                    }
            }
            __syncthreads();
            cta_jacobi(B, W, m, w, rot, pq, &flag);
            if (threadIdx.x == 0) {
                for (int a = 0; a < m; ++a) perm[a] = a;
                for (int a = 1; a < m; ++a) {
                    int v = perm[a], b = a - 1;
                    while (b >= 0 && w[perm[b]] > w[v]) { perm[b + 1] = perm[b]; --b; }
                    perm[b + 1] = v;
                }
            }
            __syncthreads();
            // X_C <- X_C W (columns in ascending eigenvalue order); rows independent
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                double2 row[RF_CMAX];
                for (int a = 0; a < m; ++a) row[a] = X[(int64_t)(c0 + a) * d.ld + r];
                for (int a = 0; a < m; ++a) {
                    double2 acc = make_double2(0.0, 0.0);
                    const int pa = perm[a];
                    for (int q = 0; q < m; ++q) acc = acc + row[q] * W[q + pa * RF_CMAX];
                    X[(int64_t)(c0 + a) * d.ld + r] = acc;
                }
            }
            for (int a = threadIdx.x; a < m; a += blockDim.x) lam[c0 + a] = w[perm[a]];
            __syncthreads();
        } else if (m > RF_CMAX) {
            if (threadIdx.x == 0) status[sid] = MMF_ST_CLUSTER;
        }
        c0 = c1;
    }
}

// ------------------------------------------------------------------ final order
// E ascending (ties by index) with the matching permutation of X's columns (into Xo).
__global__ void __launch_bounds__(256) k_sort_pairs(const MmfDesc* __restrict__ descs,
                                                    const int* __restrict__ idx,
                                                    const double* __restrict__ lamg,
                                                    const double2* __restrict__ Xg,
                                                    double* __restrict__ Eg,
                                                    double2* __restrict__ Xo) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int l = blockIdx.x;
    if (l >= n) return;
    const double* lam = lamg + d.vec_off;
    __shared__ int rank_s;
    if (threadIdx.x == 0) rank_s = 0;
    __syncthreads();
    const double v = lam[l];
    int cnt = 0;
    for (int m = threadIdx.x; m < n; m += blockDim.x) cnt += (lam[m] < v) || (lam[m] == v && m < l);
    cnt = warp_sum(cnt);
    if ((threadIdx.x & 31) == 0) atomicAdd(&rank_s, cnt);
    __syncthreads();
    const int rk = rank_s;
    if (threadIdx.x == 0) Eg[d.vec_off + rk] = v;
    const double2* src = Xg + d.mat_off + (int64_t)l * d.ld;
    double2* dst = Xo + d.mat_off + (int64_t)rk * d.ld;
    for (int r = threadIdx.x; r < n; r += blockDim.x) dst[r] = src[r];
}

// ================================================================== banded refinement step
// After one full step, the remaining corrections between eigenpairs far apart in the sorted
// order are second order in (eps |H| / gap) and negligible; the next step only forms G and S for
// pairs |i - j| <= RF_W (band storage Bm[i * (2 RF_W + 1) + (j - i + RF_W)]) and applies
// X <- X + X Et with the banded Et.
#define RF_W 16
#define RF_BW (2 * RF_W + 1)
#define RF_BC 32            // columns per CTA
#define RF_BR 16            // rows per staged chunk

__global__ void __launch_bounds__(256) k_gram_band_df32(const MmfDesc* __restrict__ descs,
                                                        const int* __restrict__ idx,
                                                        const double2* __restrict__ Xg,
                                                        const double2* __restrict__ HXg,
                                                        double2* __restrict__ Gb,
                                                        double2* __restrict__ Sb) {
    __shared__ Split xs[RF_BR][RF_BC + 2 * RF_W + 1];
    __shared__ Split hs[RF_BR][RF_BC + 2 * RF_W + 1];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int i0 = blockIdx.x * RF_BC;
    if (i0 >= n) return;
    const int cbase = i0 - RF_W;             // first staged column
    const int ncs = RF_BC + 2 * RF_W;         // staged columns
    const double2* X = Xg + d.mat_off;
    const double2* HX = HXg + d.mat_off;
    // each thread owns up to 5 (i, j) pairs: pair p = tid + 256 q, i = i0 + p / BW, j = i + p % BW - W
    DF gr[5], gi[5], sr[5], si[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) gr[q] = gi[q] = sr[q] = si[q] = DF{0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += RF_BR) {
        for (int e = threadIdx.x; e < RF_BR * ncs; e += 256) {
            const int c = e / RF_BR, kk = e - c * RF_BR;
            const int col = cbase + c, k = k0 + kk;
            const bool ok = k < n && col >= 0 && col < n;
            xs[kk][c] = split(ok ? X[(int64_t)col * d.ld + k] : make_double2(0.0, 0.0));
            hs[kk][c] = split(ok ? HX[(int64_t)col * d.ld + k] : make_double2(0.0, 0.0));
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int p = threadIdx.x + 256 * q;
            if (p < RF_BC * RF_BW) {
                const int ii = p / RF_BW, off = p - ii * RF_BW;  // column i0+ii, partner i0+ii+off-W
                const int ci = ii + RF_W, cj = ii + off;            // staged indices
                for (int kk = 0; kk < RF_BR; ++kk) {
                    df_cmacc(gr[q], gi[q], xs[kk][ci], xs[kk][cj]);
                    df_cmacc(sr[q], si[q], xs[kk][ci], hs[kk][cj]);
                }
                df_renorm(gr[q]); df_renorm(gi[q]); df_renorm(sr[q]); df_renorm(si[q]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int p = threadIdx.x + 256 * q;
        if (p < RF_BC * RF_BW) {
            const int ii = p / RF_BW, off = p - ii * RF_BW;
            const int i = i0 + ii, j = i + off - RF_W;
            if (i < n) {
                double2 g = make_double2(0.0, 0.0), s = make_double2(0.0, 0.0);
                if (j >= 0 && j < n) {
                    g = make_double2((double)gr[q].hi + (double)gr[q].lo, (double)gi[q].hi + (double)gi[q].lo);
                    s = make_double2((double)sr[q].hi + (double)sr[q].lo, (double)si[q].hi + (double)si[q].lo);
                    if (i == j) { g.y = 0.0; s.y = 0.0; }
                }
                Gb[d.mat_off + (int64_t)i * RF_BW + off] = g;
                Sb[d.mat_off + (int64_t)i * RF_BW + off] = s;
            }
        }
    }
}

// band entry (i, j) with |i - j| <= W (0 outside the matrix)
__device__ __forceinline__ double2 band_at(const double2* B, int i, int j) {
    return B[(int64_t)i * RF_BW + (j - i + RF_W)];
}

__global__ void __launch_bounds__(256) k_oa_lambda_band(const MmfDesc* __restrict__ descs,
                                                        const int* __restrict__ idx,
                                                        const double2* __restrict__ Gbg,
                                                        const double2* __restrict__ Sbg,
                                                        double* __restrict__ lamg,
                                                        int* __restrict__ cidg) {
    const MmfDesc d = descs[idx[blockIdx.x]];
    const int n = d.n;
    const double2* G = Gbg + d.mat_off;
    const double2* S = Sbg + d.mat_off;
    double* lam = lamg + d.vec_off;
    int* cid = cidg + d.vec_off;
    __shared__ double hmax;
    for (int i = threadIdx.x; i < n; i += blockDim.x) lam[i] = band_at(S, i, i).x / band_at(G, i, i).x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int i = 0; i < n; ++i) m = fmax(m, fabs(lam[i]));
        hmax = m;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        int link = 0;
        if (i + 1 < n) {
            const double gap = fabs(lam[i + 1] - lam[i]);
            const double2 num = band_at(S, i, i + 1) - lam[i + 1] * band_at(G, i, i + 1);
            link = (gap <= RF_TAU * sqrt(abs2(num))) || (gap <= 1e-13 * hmax);
        }
        cid[i] = link;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int start = 0, prev = 0;
        for (int i = 0; i < n; ++i) {
            const int link = cid[i];
            if (i == 0 || !prev) start = i;
            cid[i] = start;
            prev = link;
        }
    }
}

// Xn(:, j) = X(:, j) + sum_{|i-j|<=W} X(:, i) Et(i, j)   (Et formed on the fly from the band)
__global__ void __launch_bounds__(256) k_xe_band(const MmfDesc* __restrict__ descs,
                                                 const int* __restrict__ idx,
                                                 const double2* __restrict__ Xg,
                                                 const double2* __restrict__ Gbg,
                                                 const double2* __restrict__ Sbg,
                                                 const double* __restrict__ lamg,
                                                 const int* __restrict__ cidg,
                                                 double2* __restrict__ Xn) {
    __shared__ float2 et[RF_BW];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n;
    const int j = blockIdx.y;
    if (j >= n) return;
    const double2* G = Gbg + d.mat_off;
    const double2* S = Sbg + d.mat_off;
    const double* lam = lamg + d.vec_off;
    const int* cid = cidg + d.vec_off;
    if (threadIdx.x < RF_BW) {
        const int i = j + threadIdx.x - RF_W;
        float2 v = make_float2(0.f, 0.f);
        if (i >= 0 && i < n) {
            const double2 g = band_at(G, i, j);
            double2 e;
            if (i == j) {
                e = make_double2(0.5 * (1.0 - g.x), 0.0);
            } else {
                const double2 num = band_at(S, i, j) - lam[j] * g;
                const double gap = lam[j] - lam[i];
                const double hmax = fmax(fabs(lam[0]), fabs(lam[n - 1]));
                const bool clustered = cid[i] == cid[j] || fabs(gap) <= RF_TAU * sqrt(abs2(num)) ||
                                       fabs(gap) <= 1e-13 * fmax(hmax, fabs(lam[i]));
                e = clustered ? (-0.5) * g : (1.0 / gap) * num;
            }
            v = make_float2(__double2float_rn(e.x), __double2float_rn(e.y));
        }
        et[threadIdx.x] = v;
    }
    __syncthreads();
    const double2* X = Xg + d.mat_off;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int q = 0; q < RF_BW; ++q) {
            const int i = j + q - RF_W;
            if (i >= 0 && i < n) {
                const double2 x = X[(int64_t)i * d.ld + r];
                const float2 xf = make_float2(__double2float_rn(x.x), __double2float_rn(x.y));
                acc.x = fmaf(xf.x, et[q].x, fmaf(-xf.y, et[q].y, acc.x));
                acc.y = fmaf(xf.x, et[q].y, fmaf(xf.y, et[q].x, acc.y));
            }
        }
        const double2 x = X[(int64_t)j * d.ld + r];
        Xn[d.mat_off + (int64_t)j * d.ld + r] = make_double2(x.x + (double)acc.x, x.y + (double)acc.y);
    }
}

// The refinement is launched in three parts so that the host can time the FP64-accurate Gram
// product on its own: (1) HX = H_F X, (2) G = X^H X and S = X^H HX, (3) the rest of the full step,
// the banded step, the cluster separations and the final ordering.
cudaError_t mmf_launch_refine_pre(const MmfLaunch& L, const double2* coef, const double2* X, double2* HX) {
    if (L.count <= 0) return cudaSuccess;
    k_apply_hf<<<dim3((L.nmax + 255) / 256, (L.nmax + 15) / 16, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, coef, X, HX, 0, L.nmax);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_gram(const MmfLaunch& L, const double2* X, const double2* HX, double2* G,
                                   double2* S) {
    if (L.count <= 0) return cudaSuccess;
    const int T = (L.nmax + RF_TILE - 1) / RF_TILE;
    // the first refinement step starts from FP32 eigenvectors: X is FP32-exact
    k_gram_df32<true><<<dim3(T * (T + 1) / 2, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, HX, G, S);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_post(const MmfLaunch& L, const double2* coef, double2* X, double* E,
                                   double2* G, double2* S, double2* HX, double* lam, int* status,
                                   int* cid, int64_t mat_elems, float2* Zp, void* jobs) {
    if (L.count <= 0) return cudaSuccess;
    // rest of the full step
    k_oa_lambda<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, G, S, lam, cid);
    k_oa_etilde<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, S, lam, cid);
    // X <- X + X Et on the tensor cores (split TF32)
    k_xe_prep_B<<<dim3(512, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, S, HX);
    k_xe_prep_A<<<dim3((L.nmax + 31) / 32, (L.nmax + 31) / 32, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, X, Zp, G);
    k_xe_jobs<<<(L.count + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, L.count, Zp, G, S, HX,
                                                          (UmmaJob*)jobs);
    cudaError_t e = mmf_launch_umma(jobs, L.count, 3, L.nmax, 2 * L.nmax, 0, status, L.stream);
    if (e != cudaSuccess) return e;
    k_xe_apply<<<dim3(512, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, G);
    k_cluster_sep<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, coef, X, HX, lam, cid, status);
    // banded step
    k_apply_hf<<<dim3((L.nmax + 255) / 256, (L.nmax + 15) / 16, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, coef, X, HX, 0, L.nmax);
    k_gram_band_df32<<<dim3((L.nmax + RF_BC - 1) / RF_BC, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, X, HX, G, S);
    k_oa_lambda_band<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, G, S, lam, cid);
    k_xe_band<<<dim3((L.nmax + 255) / 256, L.nmax, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, G, S,
                                                                                lam, cid, HX);
    e = cudaMemcpyAsync(X, HX, sizeof(double2) * mat_elems, cudaMemcpyDeviceToDevice, L.stream);
    if (e != cudaSuccess) return e;
    k_cluster_sep<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, coef, X, HX, lam, cid, status);
    k_sort_pairs<<<dim3(L.nmax, L.count), 256, 0, L.stream>>>(L.desc, L.idx, lam, X, E, S);
    e = cudaMemcpyAsync(X, S, sizeof(double2) * mat_elems, cudaMemcpyDeviceToDevice, L.stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
