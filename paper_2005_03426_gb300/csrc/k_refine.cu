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
// G decides the orthogonality of the result and is formed FP64-accurately from FP32 pieces:
// every FP64 value is split x = x1 + x2 (x1 = fl32(x), x2 = fl32(x - x1)); x1*y1 is taken
// exactly (product + FMA error term), the cross terms in FP32, and the sums are accumulated in
// double-FP32 (TwoSum, Knuth 1969).  H_F X is applied in double-FP32 from the FP64 coefficients,
// never from the FP32 matrix.
// First step, residual form of S: with lam0 the eigenvalues that came with X and the residual
// W = H_F X - X diag(lam0) (FP64, small: |W| ~ eps32 |H_F|),
//     S = G diag(lam0) + C,   C = X^H W,
// so lam_i = lam0_i + c_ii / g_ii and s_ij - lam_j g_ij = c_ij - (lam_j - lam0_j) g_ij.  C only
// needs FP32 relative accuracy (its absolute error is then ~eps32^2 |H_F|) and is taken on the
// tensor cores in split TF32.  X Et only needs FP32 (Et is small) and is taken there as well.
// G itself is needed only near the diagonal: off it, g_ij enters the update of a non-clustered
// pair only through (lam_j - lam0_j) g_ij ~ eps32 |H_F| |g_ij|, negligible against c_ij there,
// and the pair's orthogonality is restored through C (c_ij - conj(c_ji) = (lam0_i - lam0_j) g_ij,
// so Et_ij + conj(Et_ji) ~ -g_ij).  Near pairs do need it: for a (near-)degenerate pair c_ij and
// (lam_j - lam0_j) g_ij are both second order in the FP32 error, and G decides whether the pair
// is clustered and gives a clustered pair's correction (keeping only the diagonal of G put a
// quasienergy of the driven lattice 3e-5 off).  Both steps therefore form G in double-FP32 on the
// band |i - j| <= RF_W only, except a full second step (below), which forms all of it.
// A second full step (large n, where one step leaves second-order errors ~(eps32 |H_F| / gap)^2
// between eigenpairs far apart in the sorted order) starts from FP64 X = X1 + Dx with
// X1 = fl32(X): G = X1^H X1 + C' + C'^H + O(|Dx|^2) with C' = X1^H Dx, the first term by the
// same double-FP32 kernel (X1 is FP32-exact), C' on the tensor cores (|Dx| ~ 2^-24 |X|).
// Below that size the second step is hybrid (below): C for all pairs and G (FP64-accurate) only
// on the band |i - j| <= RF_W, as in the first step.
// A pair is treated as clustered when |lam_i - lam_j| <= 20 |s_ij - lam_j g_ij| (the first-order
// correction would exceed 0.05) or the gap is below RF_GAMMA |H_F|; consecutive clustered indices
// form a cluster whose eigenvectors are separated by an FP64 Jacobi solve of the small
// projected matrix X_C^H H_F X_C (clusters of up to RF_CMAX vectors).  The second rule matters
// for (near-)degenerate pairs: there the gap of the Rayleigh quotients and s_ij - lam_j g_ij are
// both second order in the FP32 error, their ratio is meaningless, and a first-order correction
// taken from it ruins the pair.  RF_GAMMA = 3e-5 keeps every pair that FP32 eigenvectors cannot
// resolve well (mixing eps32 |H_F| / gap above ~2e-3) in a cluster in both steps, so that the
// first step leaves second-order errors below ~1e-5 and the second below ~1e-10.
#include <algorithm>

#include "mmf_internal.h"

#define RF_TILE 32
#define RF_KC 32
#define RF_KG 16   // k-chunk of the FP64-accurate Gram kernel
#define RF_CMAX 32
#define RF_TAU 20.0
#define RF_GAMMA 3e-5
// Band |i - j| <= RF_W of the sorted eigenpairs: the last step applies Et there in double-FP32
// (entries up to ~0.05; the first step, which another follows, in FP32), and the hybrid second
// step forms G only inside it.
#define RF_W 16
#define RF_BW (2 * RF_W + 1)
static_assert(RF_BW == MMF_REFINE_BW, "band buffer width");

// row length (floats) of the real K-major operands built from n complex entries: [Re | Im | pad]
__device__ __forceinline__ int xe_la(int n) { return (2 * n + 3) & ~3; }

// ------------------------------------------------------------------ HX = H_F X (double-FP32)
// The same product on the FP32 pipes: coefficients pre-split once per batch into FP32 pieces
// (coefs[c] = (re1, re2, im1, im2)), X as fl32(X) plus (when X is not FP32-exact) the FP32
// remainder, each complex product formed with the exact head product and FP32 cross terms,
// sums in double-FP32.  Error ~2^-48 of the sum of |terms|, far below what W = HX - X lam0
// needs (its entries are ~eps32 |H_F| and it only feeds products of FP32 relative accuracy).
__global__ void __launch_bounds__(256) k_split_coef(const double2* __restrict__ coef, float4* __restrict__ cs,
                                                    int64_t count) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < count; e += (int64_t)gridDim.x * blockDim.x) {
        const Split v = split(coef[e]);
        cs[e] = make_float4(v.r1, v.r2, v.i1, v.i2);
    }
}

// Nonzero pattern of the coefficient rows (layout with coef_matrices in mmf_internal.h): one CTA
// per system, a thread per (matrix, row).  Exact zeros only, so the sparse and dense sums agree.
__global__ void __launch_bounds__(256) k_coef_pattern(const MmfDesc* __restrict__ descs,
                                                      const int* __restrict__ idx,
                                                      const double2* __restrict__ coef, int* __restrict__ patg) {
    const MmfDesc d = descs[idx[blockIdx.x]];
    const int cap = d.pat_cap;
    if (cap <= 0) return;
    const int D = d.D, nm = coef_matrices(d);
    int* pat = patg + d.pat_off;
    int* cnt = pat + 1;
    int* jx = pat + 1 + nm * D;
    __shared__ int ok;
    if (threadIdx.x == 0) ok = 1;
    __syncthreads();
    for (int e = threadIdx.x; e < nm * D; e += blockDim.x) {
        const int m = e / D, i = e - m * D;
        const double2* A = coef + d.coef_off + (m == 0 ? 0 : (int64_t)(1 + (m - 1) / 2) * D * D);
        const bool col = m > 0 && ((m - 1) & 1);  // rows of V^dagger: columns of V
        int c = 0;
        for (int j = 0; j < D; ++j) {
            const double2 v = col ? A[j * D + i] : A[i * D + j];
            if (v.x != 0.0 || v.y != 0.0) {
                if (c < cap) jx[(int64_t)e * cap + c] = j;
                ++c;
            }
        }
        cnt[e] = c < cap ? c : cap;
        if (c > cap) ok = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) pat[0] = ok;
}

// X1 = fl32(X) and (Xlo != nullptr) Xlo = fl32(X - X1)
__global__ void __launch_bounds__(256) k_split_x(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                 const double2* __restrict__ Xg, float2* __restrict__ X1g,
                                                 float2* __restrict__ Xlog) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int64_t tot = (int64_t)d.n * d.ld;
    const double2* X = Xg + d.mat_off;
    float2* X1 = X1g + d.mat_off;
    float2* Xlo = Xlog ? Xlog + d.mat_off : nullptr;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const Split v = split(X[e]);
        X1[e] = make_float2(v.r1, v.i1);
        if (Xlo) Xlo[e] = make_float2(v.r2, v.i2);
    }
}

// acc += h x  (h from the split table, x = x1 + x2)
__device__ __forceinline__ void df_cmul_acc(DF& re, DF& im, const float4 h, float2 x1, float2 x2) {
    df_mac(re, h.x, h.y, x1.x, x2.x);
    df_mac(re, -h.z, -h.w, x1.y, x2.y);
    df_mac(im, h.x, h.y, x1.y, x2.y);
    df_mac(im, h.z, h.w, x1.x, x2.x);
}
// acc += conj(h) x
__device__ __forceinline__ void df_cmulc_acc(DF& re, DF& im, const float4 h, float2 x1, float2 x2) {
    df_mac(re, h.x, h.y, x1.x, x2.x);
    df_mac(re, h.z, h.w, x1.y, x2.y);
    df_mac(im, h.x, h.y, x1.y, x2.y);
    df_mac(im, -h.z, -h.w, x1.x, x2.x);
}

__global__ void __launch_bounds__(256) k_apply_hf_df32(const MmfDesc* __restrict__ descs,
                                                       const int* __restrict__ idx,
                                                       const float4* __restrict__ cs,
                                                       const int* __restrict__ patg,
                                                       const float2* __restrict__ X1g,
                                                       const float2* __restrict__ Xlog,
                                                       double2* __restrict__ HXg) {
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, D = d.D;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int cbeg = blockIdx.y * 16;
    if (r >= n || cbeg >= n) return;
    const int cend = min(cbeg + 16, n);
    const int b = r / D, i = r - b * D;
    int nv[MMF_MAX_MODES];
    block_nvec(d, b, nv);
    const Split shs = split(make_double2(-block_ndotw(d, b), 0.0));
    const float4 msh = make_float4(shs.r1, shs.r2, 0.f, 0.f);
    const float4* H0 = cs + d.coef_off;
    const float2* X1 = X1g + d.mat_off;
    const float2* Xlo = Xlog ? Xlog + d.mat_off : nullptr;
    const float2 z = make_float2(0.f, 0.f);
    double2* HX = HXg + d.mat_off;
    // sparse coefficient rows (the lattice's are tridiagonal): only the listed nonzeros are read
    const int* pat = patg + d.pat_off;
    const bool sp = d.pat_cap > 0 && pat[0] != 0;
    const int nm = coef_matrices(d), cap = d.pat_cap;
    const int* cnt = pat + 1;
    const int* jx = pat + 1 + nm * D;
    for (int c = cbeg; c < cend; ++c) {
        const float2* x1 = X1 + (int64_t)c * d.ld;
        const float2* x2 = Xlo ? Xlo + (int64_t)c * d.ld : nullptr;
        DF re = DF{0.f, 0.f}, im = DF{0.f, 0.f};
        // zero coefficients are skipped (exact: they add nothing)
        if (sp) {
            for (int k = 0; k < cnt[i]; ++k) {
                const int j = jx[(int64_t)i * cap + k], q = j + D * b;
                df_cmul_acc(re, im, H0[i * D + j], x1[q], x2 ? x2[q] : z);
            }
        } else {
            for (int j = 0; j < D; ++j) {
                const float4 h = H0[i * D + j];
                if (h.x == 0.f && h.z == 0.f) continue;
                const int q = j + D * b;
                df_cmul_acc(re, im, h, x1[q], x2 ? x2[q] : z);
            }
        }
        df_cmul_acc(re, im, msh, x1[r], x2 ? x2[r] : z);
        int64_t off = d.coef_off + (int64_t)D * D;
        int m = 1;
        for (int l = 0; l < d.K; ++l) {
            for (int h = 1; h <= d.nharm[l]; ++h, m += 2) {
                const float4* V = cs + off + (int64_t)(h - 1) * D * D;
                if (nv[l] + h <= d.N[l]) {
                    const int bu = b + h * d.S[l];
                    if (sp) {
                        const int e = m * D + i;
                        for (int k = 0; k < cnt[e]; ++k) {
                            const int j = jx[(int64_t)e * cap + k], q = j + D * bu;
                            df_cmul_acc(re, im, V[i * D + j], x1[q], x2 ? x2[q] : z);
                        }
                    } else {
                        for (int j = 0; j < D; ++j) {
                            const float4 hv = V[i * D + j];
                            if (hv.x == 0.f && hv.z == 0.f) continue;
                            const int q = j + D * bu;
                            df_cmul_acc(re, im, hv, x1[q], x2 ? x2[q] : z);
                        }
                    }
                }
                if (nv[l] - h >= -d.N[l]) {
                    const int bd = b - h * d.S[l];
                    if (sp) {
                        const int e = (m + 1) * D + i;
                        for (int k = 0; k < cnt[e]; ++k) {
                            const int j = jx[(int64_t)e * cap + k], q = j + D * bd;
                            df_cmulc_acc(re, im, V[j * D + i], x1[q], x2 ? x2[q] : z);
                        }
                    } else {
                        for (int j = 0; j < D; ++j) {
                            const float4 hv = V[j * D + i];
                            if (hv.x == 0.f && hv.z == 0.f) continue;
                            const int q = j + D * bd;
                            df_cmulc_acc(re, im, hv, x1[q], x2 ? x2[q] : z);
                        }
                    }
                }
            }
            off += (int64_t)d.nharm[l] * D * D;
        }
        HX[(int64_t)c * d.ld + r] = df_value(re, im);
    }
}

// ------------------------------------------------------------------ G = X1^H X1 (double-FP32)
// X1 = fl32(X) in its own FP32 buffer (written once by k_split_x), so the kernel converts
// nothing: each conj(a) b of FP32 values is accumulated exactly (product + FMA error term) into
// a double-FP32 sum.  Upper-triangle tiles (I <= J) of 32 x 32; both triangles are written.
__global__ void __launch_bounds__(256) k_gram_x1(const MmfDesc* __restrict__ descs,
                                                 const int* __restrict__ idx,
                                                 const float2* __restrict__ X1g,
                                                 double2* __restrict__ Gg) {
    __shared__ float2 xi[RF_KG][RF_TILE + 1];
    __shared__ float2 xj[RF_KG][RF_TILE + 1];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int T = (n + RF_TILE - 1) / RF_TILE;
    // tile index -> (I, J), I <= J
    int t = blockIdx.x, I = 0;
    if (t >= T * (T + 1) / 2) return;
    while (t >= T - I) { t -= T - I; ++I; }
    const int J = I + t;
    const int i0 = I * RF_TILE, j0 = J * RF_TILE;
    const float2* X = X1g + d.mat_off;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;  // outputs (ty + 16a, tx + 16b)
    DF gr[2][2], gi[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) gr[a][b] = gi[a][b] = DF{0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += RF_KG) {
        for (int e = threadIdx.x; e < RF_KG * RF_TILE; e += 256) {
            const int c = e / RF_KG, kk = e - c * RF_KG;
            const int k = k0 + kk;
            const float2 z = make_float2(0.f, 0.f);
            xi[kk][c] = (k < n && i0 + c < n) ? X[(int64_t)(i0 + c) * d.ld + k] : z;
            xj[kk][c] = (k < n && j0 + c < n) ? X[(int64_t)(j0 + c) * d.ld + k] : z;
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < RF_KG; ++kk) {
            const float2 a[2] = {xi[kk][ty], xi[kk][ty + 16]};
            const float2 b[2] = {xj[kk][tx], xj[kk][tx + 16]};
#pragma unroll
            for (int p = 0; p < 2; ++p)
#pragma unroll
                for (int q = 0; q < 2; ++q) {  // conj(a) b
                    df_mac11(gr[p][q], a[p].x, b[q].x);
                    df_mac11(gr[p][q], a[p].y, b[q].y);
                    df_mac11(gi[p][q], a[p].x, b[q].y);
                    df_mac11(gi[p][q], -a[p].y, b[q].x);
                }
        }
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                df_renorm(gr[a][b]);
                df_renorm(gi[a][b]);
            }
        __syncthreads();
    }
    double2* G = Gg + d.mat_off;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int i = i0 + ty + 16 * a, j = j0 + tx + 16 * b;
            if (i < n && j < n && (I < J || i <= j)) {
                double2 g = df_value(gr[a][b], gi[a][b]);
                if (i == j) g.y = 0.0;
                G[(int64_t)j * d.ld + i] = g;
                G[(int64_t)i * d.ld + j] = conj(g);
            }
        }
}

// ------------------------------------------------------------------ C = X^H W on tensor cores
// Re C = Xr^T Wr + Xi^T Wi and Im C = Xr^T Wi - Xi^T Wr as one real product over K = 2n:
//   A row i = [Re x_i | Im x_i],  B row j = [Re w_j | Im w_j] (j < n), [Im w_j | -Re w_j] (n + j),
//   C row i = [Re c_i. | Im c_i.]   (x_i, w_j columns of X and W),
// in split TF32 (three products) by k_tf3_gemm.  The operands are written pre-tiled (hi and lo
// pieces, zero padding) into the system's operand area (ops: A, then B); C goes to T.  For X in
// FP64 (second step) A holds the split of fl32(X).
__device__ __forceinline__ float* tf3_area(void* pool, const MmfDesc& d) {
    return reinterpret_cast<float*>(reinterpret_cast<uint16_t*>(pool) + d.oz_off);
}
__device__ __forceinline__ void tf3_put(float* P, int rows, int K, int r, int k, float v) {
    const float v1 = tf32_round(v);
    P[tf3_pos(rows, K, 0, r, k)] = v1;
    P[tf3_pos(rows, K, 1, r, k)] = tf32_round(v - v1);
}

// B (2n x 2n) from W = HX - X diag(lam0) (FP64, rounded once to FP32)
__global__ void __launch_bounds__(256) k_w_prep_B(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx,
                                                  const double2* __restrict__ Xg,
                                                  const double2* __restrict__ HXg,
                                                  const double* __restrict__ lam0g, void* __restrict__ pool) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, K = 2 * n;
    const int rp = tf3_nq(2 * n) * 128, kp = tf3_nt(K) * 32;
    const double2* X = Xg + d.mat_off;
    const double2* HX = HXg + d.mat_off;
    const double* lam0 = lam0g + d.vec_off;
    float* B = tf3_area(pool, d) + 2 * tf3_piece(n, K);
    // each complex entry w = W(kk, jj) once (FP64), written as its four real entries
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int jj = (int)(e / n), kk = (int)(e - (int64_t)jj * n);
        const int64_t o = (int64_t)jj * d.ld + kk;
        const double2 w = HX[o] - lam0[jj] * X[o];
        const float wr = (float)w.x, wi = (float)w.y;
        tf3_put(B, 2 * n, K, jj, kk, wr);
        tf3_put(B, 2 * n, K, jj, n + kk, wi);
        tf3_put(B, 2 * n, K, n + jj, kk, wi);
        tf3_put(B, 2 * n, K, n + jj, n + kk, -wr);
    }
    // zeros: K padding of every row, and the padding rows
    const int kpad = kp - K;
    const int64_t tz = (int64_t)rp * kpad + (int64_t)(rp - 2 * n) * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tz; e += (int64_t)gridDim.x * blockDim.x) {
        int j, k;
        if (e < (int64_t)rp * kpad) {
            j = (int)(e / kpad);
            k = K + (int)(e - (int64_t)j * kpad);
        } else {
            const int64_t f = e - (int64_t)rp * kpad;
            j = 2 * n + (int)(f / K);
            k = (int)(f - (int64_t)(j - 2 * n) * K);
        }
        tf3_put(B, 2 * n, K, j, k, 0.f);
    }
}

// A (n x 2n): row i = [Re x_i | Im x_i] of X1 = fl32(X)
__global__ void __launch_bounds__(256) k_w_prep_A(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx,
                                                  const float2* __restrict__ X1g, void* __restrict__ pool) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, K = 2 * n;
    const int rp = tf3_nq(n) * 128, kp = tf3_nt(K) * 32;
    const float2* X = X1g + d.mat_off;
    float* A = tf3_area(pool, d);
    const int64_t tot = (int64_t)rp * kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / kp), k = (int)(e - (int64_t)i * kp);
        float v = 0.f;
        if (i < n && k < K) {
            const float2 x = X[(int64_t)i * d.ld + (k < n ? k : k - n)];
            v = k < n ? x.x : x.y;
        }
        tf3_put(A, n, K, i, k, v);
    }
}

// B rows for C' = X1^H Dx: [Re dx_j | Im dx_j] (j < n), [Im dx_j | -Re dx_j] (n + j), with
// Dx = X - fl32(X) (exact in FP64)
__global__ void __launch_bounds__(256) k_d_prep_B(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx,
                                                  const double2* __restrict__ Xg, void* __restrict__ pool) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, K = 2 * n;
    const int rp = tf3_nq(2 * n) * 128, kp = tf3_nt(K) * 32;
    const double2* X = Xg + d.mat_off;
    float* B = tf3_area(pool, d) + 2 * tf3_piece(n, K);
    const int64_t tot = (int64_t)rp * kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / kp), k = (int)(e - (int64_t)j * kp);
        float v = 0.f;
        if (j < 2 * n && k < K) {
            const int jj = j < n ? j : j - n, kk = k < n ? k : k - n;
            const double2 x = X[(int64_t)jj * d.ld + kk];
            const double2 dx = make_double2(x.x - (double)(float)x.x, x.y - (double)(float)x.y);
            double r;
            if (j < n) r = (k < n) ? dx.x : dx.y;
            else r = (k < n) ? dx.y : -dx.x;
            v = (float)r;
        }
        tf3_put(B, 2 * n, K, j, k, v);
    }
}

// one job per system: A and B from the operand area, C at float offset (second ? 2 n^2 : 0) of
// the system's T slot
__global__ void k_w_jobs(const MmfDesc* __restrict__ descs, const int* __restrict__ idx, int count, void* pool,
                         double2* T, int second_c, Tf3Job* jobs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const MmfDesc d = descs[idx[i]];
    const int n = d.n;
    Tf3Job j;
    j.A = tf3_area(pool, d);
    j.B = j.A + 2 * tf3_piece(n, 2 * n);
    j.C = reinterpret_cast<float*>(T + d.mat_off) + (second_c ? (int64_t)2 * n * n : 0);
    j.M = n; j.N = 2 * n; j.K = 2 * n; j.ldc = 2 * n;
    j.mode = TF3_STORE;
    jobs[i] = j;
}

// G <- G + C' + C'^H (both triangles; C' row i = [Re c'_i. | Im c'_i.])
__global__ void __launch_bounds__(256) k_gram_fix(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx, double2* __restrict__ Gg,
                                                  const double2* __restrict__ Tg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    double2* G = Gg + d.mat_off;
    const float* Cp = reinterpret_cast<const float*>(Tg + d.mat_off) + (int64_t)2 * n * n;
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / n), i = (int)(e - (int64_t)j * n);
        const double re = (double)Cp[(int64_t)i * 2 * n + j] + (double)Cp[(int64_t)j * 2 * n + i];
        const double im = (double)Cp[(int64_t)i * 2 * n + n + j] - (double)Cp[(int64_t)j * 2 * n + n + i];
        double2& g = G[(int64_t)j * d.ld + i];
        g = make_double2(g.x + re, i == j ? 0.0 : g.y + im);
    }
}

// ------------------------------------------------------------------ lam, clusters
// C = X^H W from the tensor cores, at the start of the system's slot of the T buffer: row i holds
// Re c_i. (n floats) then Im c_i. (n floats).  C' (second full step) follows it.
__device__ __forceinline__ double2 c_entry(const float* C, int n, int i, int j) {
    return make_double2((double)C[(int64_t)i * 2 * n + j], (double)C[(int64_t)i * 2 * n + n + j]);
}
// s_ij - lam_j g_ij in the residual form, with dl_j = lam_j - lam0_j = c_jj / g_jj
__device__ __forceinline__ double2 oa_num(const float* C, int n, int i, int j, double2 g, double dl_j) {
    return c_entry(C, n, i, j) - dl_j * g;
}

// One CTA per system: lam_i = lam0_i + c_ii / g_ii; link_i = pair (i, i+1) clustered; cluster
// id = the first index of its run.  aux per system: cid (n ints) stored in the E2 buffer's tail.
__global__ void __launch_bounds__(256) k_oa_lambda(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Gg,
                                                   const double2* __restrict__ Cg,
                                                   const double* __restrict__ lam0g,
                                                   double* __restrict__ lamg,
                                                   int* __restrict__ cidg) {
    const MmfDesc d = descs[idx[blockIdx.x]];
    const int n = d.n;
    const double2* G = Gg + d.mat_off;
    const float* C = reinterpret_cast<const float*>(Cg + d.mat_off);
    const double* lam0 = lam0g + d.vec_off;
    double* lam = lamg + d.vec_off;
    int* cid = cidg + d.vec_off;
    __shared__ double hmax;
    for (int i = threadIdx.x; i < n; i += blockDim.x)
        lam[i] = lam0[i] + (double)C[(int64_t)i * 2 * n + i] / G[(int64_t)i * d.ld + i].x;
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
            const double2 num = oa_num(C, n, i, i + 1, G[(int64_t)(i + 1) * d.ld + i], lam[i + 1] - lam0[i + 1]);
            link = (gap <= RF_TAU * sqrt(abs2(num))) || (gap <= RF_GAMMA * hmax);
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

// Et in place of G (diagonal and clustered pairs: r/2; others: OA formula).  One 32 x 32 tile
// (rows i, columns j) per block iteration: G is column-major (i contiguous) and C row-major
// (j contiguous), so C's tile is read along j into shared memory first and both are then used
// with i fastest across the threads.  g_band: G was formed only on the band |i - j| <= RF_W and
// is taken as 0 off it (its entries there are not read and need not be set).
__global__ void __launch_bounds__(256) k_oa_etilde(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   double2* __restrict__ Gg,
                                                   const double2* __restrict__ Cg,
                                                   const double* __restrict__ lam0g,
                                                   const double* __restrict__ lamg,
                                                   const int* __restrict__ cidg, int g_band) {
    __shared__ float cre[32][33], cim[32][33];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    double2* G = Gg + d.mat_off;
    const float* C = reinterpret_cast<const float*>(Cg + d.mat_off);
    const double* lam0 = lam0g + d.vec_off;
    const double* lam = lamg + d.vec_off;
    const int* cid = cidg + d.vec_off;
    double hmax = fmax(fabs(lam[0]), fabs(lam[n - 1]));
    const float tiny = (float)(RF_GAMMA * hmax);  // |lam_i| <= hmax (ascending order)
    const int nt = (n + 31) / 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int tile = blockIdx.x; tile < nt * nt; tile += gridDim.x) {
        const int i0 = (tile % nt) * 32, j0 = (tile / nt) * 32;
        __syncthreads();  // the previous tile's reads of cre / cim are done
        for (int q = ty; q < 32; q += 8) {  // C(i0 + q, j0 + tx): j contiguous
            const int i = i0 + q, j = j0 + tx;
            const bool ok = i < n && j < n;
            cre[q][tx] = ok ? C[(int64_t)i * 2 * n + j] : 0.f;
            cim[q][tx] = ok ? C[(int64_t)i * 2 * n + n + j] : 0.f;
        }
        __syncthreads();
        const int i = i0 + tx;
        if (i >= n) continue;
        const double lami = lam[i];
        const int cidi = cid[i];
        for (int q = ty; q < 32; q += 8) {
            const int j = j0 + q;
            if (j >= n) break;
            const int64_t o = (int64_t)j * d.ld + i;
            const double2 g = (g_band && abs(i - j) > RF_W) ? make_double2(0.0, 0.0) : G[o];
            double2 et;
            if (i == j) {
                et = make_double2(0.5 * (1.0 - g.x), 0.0);
            } else if (abs(i - j) <= RF_W) {
                // the band is applied in double-FP32: FP64 here
                const double2 num = oa_num(C, n, i, j, g, lam[j] - lam0[j]);
                const double gap = lam[j] - lami;
                const bool clustered = cidi == cid[j] || gap * gap <= RF_TAU * RF_TAU * abs2(num) ||
                                       fabs(gap) <= RF_GAMMA * fmax(hmax, fabs(lami));
                et = clustered ? (-0.5) * g : (1.0 / gap) * num;
            } else {
                // off the band Et goes through the split-TF32 product (FP32 accuracy): FP32 here,
                // with the gap taken in FP64 before rounding
                const float gx = (float)g.x, gy = (float)g.y;
                const float dl = (float)(lam[j] - lam0[j]);
                const float nr = cre[tx][q] - dl * gx, ni = cim[tx][q] - dl * gy;
                const float gap = (float)(lam[j] - lami);
                const bool clustered = cidi == cid[j] || gap * gap <= (float)(RF_TAU * RF_TAU) * (nr * nr + ni * ni) ||
                                       fabsf(gap) <= tiny;
                const float r = 1.f / gap;
                et = clustered ? make_double2(-0.5 * g.x, -0.5 * g.y) : make_double2(nr * r, ni * r);
            }
            G[o] = et;
        }
    }
}

// ------------------------------------------------------------------ Xn = X + X Et on tensor cores
// The complex product is a real product of twice the size,
//   [Re Y | Im Y] = [Re X, Im X] [[Re E, Im E], [-Im E, Re E]],
// taken on the tcgen05 engine in split TF32 (x = x1 + x2, x1 = tf32(x), x2 = tf32(x - x1);
// x y ~ x1 y1 + x1 y2 + x2 y1, about FP32 accuracy) for the entries of Et outside the band
// |i - j| <= RF_W, which are small (|Et_ij| ~ eps32 |H_F| / gap_ij), so that the FP32 error
// stays far below the target.  The band, where Et reaches ~0.05 for close pairs, is applied in
// double-FP32 on the SIMT units (k_et_band, k_xe_apply).  The operands are written pre-tiled
// into the system's operand area (as for C = X^H W); C (n x 2n) goes to the Et buffer after B
// has been built from it.
__global__ void __launch_bounds__(256) k_xe_prep_B(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const double2* __restrict__ Etg, void* __restrict__ pool) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, K = 2 * n;
    const int rp = tf3_nq(2 * n) * 128, kp = tf3_nt(K) * 32;
    const double2* Et = Etg + d.mat_off;
    float* B = tf3_area(pool, d) + 2 * tf3_piece(n, K);
    // each complex entry Et(kk, jj) once, written as its four real entries (0 on the band)
    const int64_t tot = (int64_t)n * n;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int jj = (int)(e / n), kk = (int)(e - (int64_t)jj * n);
        float xr = 0.f, xi = 0.f;
        if (abs(jj - kk) > RF_W) {  // the band is applied in double-FP32 by k_xe_apply
            const double2 x = Et[(int64_t)jj * d.ld + kk];
            xr = (float)x.x;
            xi = (float)x.y;
        }
        tf3_put(B, 2 * n, K, jj, kk, xr);
        tf3_put(B, 2 * n, K, jj, n + kk, -xi);
        tf3_put(B, 2 * n, K, n + jj, kk, xi);
        tf3_put(B, 2 * n, K, n + jj, n + kk, xr);
    }
    // zeros: K padding of every row, and the padding rows
    const int kpad = kp - K;
    const int64_t tz = (int64_t)rp * kpad + (int64_t)(rp - 2 * n) * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tz; e += (int64_t)gridDim.x * blockDim.x) {
        int j, k;
        if (e < (int64_t)rp * kpad) {
            j = (int)(e / kpad);
            k = K + (int)(e - (int64_t)j * kpad);
        } else {
            const int64_t f = e - (int64_t)rp * kpad;
            j = 2 * n + (int)(f / K);
            k = (int)(f - (int64_t)(j - 2 * n) * K);
        }
        tf3_put(B, 2 * n, K, j, k, 0.f);
    }
}

// A (n x 2n): row r = [Re X(r, :) | Im X(r, :)] of X1, transposed through shared memory in 32 x 32
// blocks; the grid covers the padded rows, and the blocks of the last column block also zero
// the K padding.
__global__ void __launch_bounds__(256) k_xe_prep_A(const MmfDesc* __restrict__ descs,
                                                   const int* __restrict__ idx,
                                                   const float2* __restrict__ X1g, void* __restrict__ pool) {
    __shared__ float2 t[32][33];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, K = 2 * n;
    const int rp = tf3_nq(n) * 128, kp = tf3_nt(K) * 32;
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    if (r0 >= rp || c0 >= n) return;
    const float2* X = X1g + d.mat_off;
    float* A = tf3_area(pool, d);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int q = ty; q < 32; q += 8) {  // X(r0 + tx, c0 + q), rows fastest
        const int r = r0 + tx, c = c0 + q;
        t[q][tx] = (r < n && c < n) ? X[(int64_t)c * d.ld + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {  // A(r0 + q, c0 + tx) = Re, A(r0 + q, n + c0 + tx) = Im
        const int r = r0 + q, c = c0 + tx;
        if (c < n) {
            const float2 x = t[tx][q];
            tf3_put(A, n, K, r, c, x.x);
            tf3_put(A, n, K, r, n + c, x.y);
        }
        if (c0 + 32 >= n && 2 * n + tx < kp) tf3_put(A, n, K, r, 2 * n + tx, 0.f);  // K padding
    }
}

__global__ void k_xe_jobs(const MmfDesc* __restrict__ descs, const int* __restrict__ idx, int count, void* pool,
                          double2* R, Tf3Job* jobs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const MmfDesc d = descs[idx[i]];
    const int n = d.n, la = xe_la(n);
    Tf3Job j;
    j.A = tf3_area(pool, d);
    j.B = j.A + 2 * tf3_piece(n, 2 * n);
    j.C = reinterpret_cast<float*>(R + d.mat_off) + (int64_t)n * la;
    j.M = n; j.N = 2 * n; j.K = 2 * n; j.ldc = 2 * n;
    j.mode = TF3_STORE;
    jobs[i] = j;
}

// the band of Et, Eb[i * RF_BW + (j - i + RF_W)] = Et(i, j) (0 outside the matrix), saved before
// the Et buffer is reused for the tensor-core operands
__global__ void __launch_bounds__(256) k_et_band(const MmfDesc* __restrict__ descs,
                                                 const int* __restrict__ idx,
                                                 const double2* __restrict__ Etg,
                                                 double2* __restrict__ Ebg) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const double2* Et = Etg + d.mat_off;
    double2* Eb = Ebg + (int64_t)d.vec_off * RF_BW;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n * RF_BW; e += gridDim.x * blockDim.x) {
        const int i = e / RF_BW, j = i + (e - i * RF_BW) - RF_W;
        Eb[e] = (j >= 0 && j < n) ? Et[(int64_t)j * d.ld + i] : make_double2(0.0, 0.0);
    }
}

// Xn(:, j) = X(:, j) + C(:, j) + sum_{|i-j|<=W} X(:, i) Et(i, j): C from the tensor cores (Et
// outside the band), the band in double-FP32 from X1 = fl32(X) (exact in the first step; in a
// second step the remainder times Et is below 2^-24 |Et| and dropped) and Et split in two FP32
// pieces, or in plain FP32 where every band entry of the tile is below XT_SMALL (a second step's
// corrections) or where a further full step follows (band_fp32): the FP32 band then adds an
// error of at most ~RF_BW x 2^-24 x 0.05 ~ 1e-7 (typically ~1e-8) to the columns of Xn, below
// the second-order error ~1e-5 the step leaves between close pairs, and the next step, which
// forms G and C from Xn itself, removes both.  Xn overwrites X in place: the band reads the
// neighbouring columns from X1, and each thread reads only the element of X it writes.
// One CTA per XT_R x XT_C tile of Xn: the XT_C + 2W neighbouring columns of X1, the band of Et
// and the tile of C are staged in shared memory; thread (row, group of XT_CPT columns).
#define XT_R 32
#define XT_C 32
#define XT_SMALL 1e-7f  // band entries below this go through plain FP32
#define XT_CPT (XT_C * XT_R / 256)   // output columns per thread
__global__ void __launch_bounds__(256) k_xe_apply(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx, double2* Xg,
                                                  const float2* __restrict__ X1g, const double2* __restrict__ R,
                                                  const double2* __restrict__ Ebg, int band_fp32) {
    __shared__ float2 xs[XT_C + 2 * RF_W][XT_R];
    __shared__ Split es[RF_BW][XT_C];
    __shared__ float cs[2][XT_R][XT_C + 1];
    __shared__ int big;
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n, la = xe_la(n);
    if (threadIdx.x == 0) big = 0;
    __syncthreads();
    const int r0 = blockIdx.x * XT_R, j0 = blockIdx.y * XT_C;
    if (r0 >= n || j0 >= n) return;
    const double2* Eb = Ebg + (int64_t)d.vec_off * RF_BW;
    const float* C = reinterpret_cast<const float*>(R + d.mat_off) + (int64_t)n * la;
    const float2* X1 = X1g + d.mat_off;
    for (int e = threadIdx.x; e < (XT_C + 2 * RF_W) * XT_R; e += 256) {
        const int cc = e / XT_R, rr = e - cc * XT_R, col = j0 - RF_W + cc, row = r0 + rr;
        xs[cc][rr] = (col >= 0 && col < n && row < n) ? X1[(int64_t)col * d.ld + row] : make_float2(0.f, 0.f);
    }
    bool bigl = false;
    for (int e = threadIdx.x; e < RF_BW * XT_C; e += 256) {
        const int q = e / XT_C, c = e - q * XT_C, j = j0 + c, i = j + q - RF_W;
        const Split v = split((j < n && i >= 0 && i < n) ? Eb[(int64_t)i * RF_BW + (j - i + RF_W)] : make_double2(0.0, 0.0));
        es[q][c] = v;
        bigl |= fmaxf(fabsf(v.r1), fabsf(v.i1)) > XT_SMALL;
    }
    if (__any_sync(0xffffffffu, bigl) && (threadIdx.x & 31) == 0) big = 1;
    for (int e = threadIdx.x; e < XT_R * XT_C; e += 256) {
        const int rr = e / XT_C, c = e - rr * XT_C, row = r0 + rr, j = j0 + c;
        const bool ok = row < n && j < n;
        cs[0][rr][c] = ok ? C[(int64_t)row * 2 * n + j] : 0.f;
        cs[1][rr][c] = ok ? C[(int64_t)row * 2 * n + n + j] : 0.f;
    }
    __syncthreads();
    const int rr = threadIdx.x & (XT_R - 1), cg = threadIdx.x / XT_R;
    const int r = r0 + rr;
    if (r >= n) return;
    double2* X = Xg + d.mat_off;
    if (!big || band_fp32) {
        // every band entry of the tile is below XT_SMALL (a second step's corrections): plain
        // FP32, whose error (about 33 x 2^-24 x XT_SMALL for |X| <= 1) stays near 2e-13 at most;
        // or a full step follows, which removes the FP32 error of this one
#pragma unroll 1
        for (int c = cg * XT_CPT; c < cg * XT_CPT + XT_CPT; ++c) {
            const int j = j0 + c;
            if (j >= n) break;
            float ar = 0.f, ai = 0.f;
#pragma unroll 11
            for (int q = 0; q < RF_BW; ++q) {
                const float2 x = xs[c + q][rr];
                const Split e = es[q][c];
                ar = fmaf(x.x, e.r1, fmaf(-x.y, e.i1, ar));
                ai = fmaf(x.x, e.i1, fmaf(x.y, e.r1, ai));
            }
            const double2 x = X[(int64_t)j * d.ld + r];
            X[(int64_t)j * d.ld + r] =
                make_double2(x.x + ((double)cs[0][rr][c] + (double)ar), x.y + ((double)cs[1][rr][c] + (double)ai));
        }
        return;
    }
#pragma unroll 1
    for (int c = cg * XT_CPT; c < cg * XT_CPT + XT_CPT; ++c) {
        const int j = j0 + c;
        if (j >= n) break;
        DF ar = DF{0.f, 0.f}, ai = DF{0.f, 0.f};
#pragma unroll 11
        for (int q = 0; q < RF_BW; ++q) {  // zero outside the matrix (staged as zeros)
            const float2 x = xs[c + q][rr];
            const Split e = es[q][c];
            df_mac1(ar, x.x, e.r1, e.r2);
            df_mac1(ar, -x.y, e.i1, e.i2);
            df_mac1(ai, x.x, e.i1, e.i2);
            df_mac1(ai, x.y, e.r1, e.r2);
        }
        const double2 band = df_value(ar, ai);
        const double2 x = X[(int64_t)j * d.ld + r];
        X[(int64_t)j * d.ld + r] =
            make_double2(x.x + ((double)cs[0][rr][c] + band.x), x.y + ((double)cs[1][rr][c] + band.y));
    }
}

// ------------------------------------------------------------------ cluster separation
// Clusters are independent: each CTA of a system takes every gridDim.x-th candidate first index.
// For cluster C (m vectors), Rayleigh-Ritz on span(X_C) in FP64:
// B = X_C^H H_F X_C (H_F X_C from the HX buffer, recomputed for the new X) and
// G_C = X_C^H X_C = L L^H (Cholesky); B' = L^-1 B L^-H, X_C <- X_C L^-H (orthonormal columns);
// cyclic Jacobi on B', X_C <- X_C W, lam_C <- eigenvalues of B' ascending.  Without the
// G_C factor the eigenvalues of B would carry an error |lam| |G_C - I|, and after the hybrid
// second step a cluster's columns are orthonormal only to ~1e-10 (the pair's Et is r/2, first
// order), which is the size of the separation of the near-degenerate pairs the cluster holds.
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
                                                     const int* __restrict__ patg,
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
    const int sid = idx[blockIdx.y];
    const MmfDesc d = descs[sid];
    const int n = d.n, D = d.D;
    double2* X = Xg + d.mat_off;
    double2* HX = HXg + d.mat_off;
    double* lam = lamg + d.vec_off;
    const int* cid = cidg + d.vec_off;
    const double2* H0 = coef + d.coef_off;
    const int* pat = patg + d.pat_off;
    const bool sp = d.pat_cap > 0 && pat[0] != 0;
    const int nm = coef_matrices(d), cap = d.pat_cap;
    const int* cnt = pat + 1;
    const int* jx = pat + 1 + nm * D;
    // clusters are disjoint: the CTAs of a system take them in parallel (c0 = first index)
    for (int c0 = blockIdx.x; c0 < n; c0 += gridDim.x) {
        if (cid[c0] != c0 || c0 + 1 >= n || cid[c0 + 1] != c0) continue;
        int c1 = c0 + 2;
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
                if (sp) {
                    for (int k = 0; k < cnt[i]; ++k) {
                        const int j = jx[(int64_t)i * cap + k];
                        acc = acc + H0[i * D + j] * x[j + D * b];
                    }
                } else {
                    for (int j = 0; j < D; ++j) {
                        const double2 h = H0[i * D + j];
                        if (h.x != 0.0 || h.y != 0.0) acc = acc + h * x[j + D * b];
                    }
                }
                acc = acc - block_ndotw(d, b) * x[r];
                int64_t off = d.coef_off + (int64_t)D * D;
                int mq = 1;
                for (int l = 0; l < d.K; ++l) {
                    for (int h = 1; h <= d.nharm[l]; ++h, mq += 2) {
                        const double2* V = coef + off + (int64_t)(h - 1) * D * D;
                        if (nv[l] + h <= d.N[l]) {
                            const double2* xu = x + D * (b + h * d.S[l]);
                            if (sp) {
                                const int e2 = mq * D + i;
                                for (int k = 0; k < cnt[e2]; ++k) {
                                    const int j = jx[(int64_t)e2 * cap + k];
                                    acc = acc + V[i * D + j] * xu[j];
                                }
                            } else {
                                for (int j = 0; j < D; ++j) {
                                    const double2 v = V[i * D + j];
                                    if (v.x != 0.0 || v.y != 0.0) acc = acc + v * xu[j];
                                }
                            }
                        }
                        if (nv[l] - h >= -d.N[l]) {
                            const double2* xd = x + D * (b - h * d.S[l]);
                            if (sp) {
                                const int e2 = (mq + 1) * D + i;
                                for (int k = 0; k < cnt[e2]; ++k) {
                                    const int j = jx[(int64_t)e2 * cap + k];
                                    acc = acc + cmulc(V[j * D + i], xd[j]);
                                }
                            } else {
                                for (int j = 0; j < D; ++j) {
                                    const double2 v = V[j * D + i];
                                    if (v.x != 0.0 || v.y != 0.0) acc = acc + cmulc(v, xd[j]);
                                }
                            }
                        }
                    }
                    off += (int64_t)d.nharm[l] * D * D;
                }
                HX[(int64_t)c * d.ld + r] = acc;
            }
            __syncthreads();
            // B = X_C^H HX_C and G_C = X_C^H X_C (into W), one warp per entry
            for (int e = threadIdx.x >> 5; e < m * m; e += blockDim.x >> 5) {
                const int p = e % m, q = e / m;
                const double2* xp = X + (int64_t)(c0 + p) * d.ld;
                const double2* xq = X + (int64_t)(c0 + q) * d.ld;
                const double2* hq = HX + (int64_t)(c0 + q) * d.ld;
                double2 acc = make_double2(0.0, 0.0), gac = make_double2(0.0, 0.0);
                for (int r = threadIdx.x & 31; r < n; r += 32) {
                    acc = acc + cmulc(xp[r], hq[r]);
                    gac = gac + cmulc(xp[r], xq[r]);
                }
                acc.x = warp_sum(acc.x);
                acc.y = warp_sum(acc.y);
                gac.x = warp_sum(gac.x);
                gac.y = warp_sum(gac.y);
                if ((threadIdx.x & 31) == 0) {
                    B[p + q * RF_CMAX] = acc;
                    W[p + q * RF_CMAX] = gac;
                }
            }
            __syncthreads();
            // L (lower, in W) with G_C = L L^H; a non-positive pivot (columns not independent
            // to FP64) leaves the cluster without the G_C factor (L = I)
            if (threadIdx.x == 0) {
                int ok = 1;
                for (int j = 0; j < m && ok; ++j) {
                    double s = W[j + j * RF_CMAX].x;
                    for (int k = 0; k < j; ++k) s -= abs2(W[j + k * RF_CMAX]);
                    if (!(s > 0.0)) { ok = 0; break; }
                    const double ljj = sqrt(s);
                    W[j + j * RF_CMAX] = make_double2(ljj, 0.0);
                    for (int i = j + 1; i < m; ++i) {
                        double2 a = W[i + j * RF_CMAX];
                        for (int k = 0; k < j; ++k) a = a - W[i + k * RF_CMAX] * conj(W[j + k * RF_CMAX]);
                        W[i + j * RF_CMAX] = (1.0 / ljj) * a;
                    }
                }
                if (!ok)
                    for (int j = 0; j < m; ++j)
                        for (int i = j; i < m; ++i) W[i + j * RF_CMAX] = make_double2(i == j ? 1.0 : 0.0, 0.0);
            }
            __syncthreads();
            // B <- L^-1 B: forward substitution, one column per thread
            for (int t = threadIdx.x; t < m; t += blockDim.x)
                for (int i = 0; i < m; ++i) {
                    double2 a = B[i + t * RF_CMAX];
                    for (int k = 0; k < i; ++k) a = a - W[i + k * RF_CMAX] * B[k + t * RF_CMAX];
                    B[i + t * RF_CMAX] = (1.0 / W[i + i * RF_CMAX].x) * a;
                }
            __syncthreads();
            // B <- B L^-H: row t solves y L^H = B[t, :] (y_j = (b_j - sum_k<j y_k conj(L_jk)) / L_jj)
            for (int t = threadIdx.x; t < m; t += blockDim.x)
                for (int j = 0; j < m; ++j) {
                    double2 a = B[t + j * RF_CMAX];
                    for (int k = 0; k < j; ++k) a = a - B[t + k * RF_CMAX] * conj(W[j + k * RF_CMAX]);
                    B[t + j * RF_CMAX] = (1.0 / W[j + j * RF_CMAX].x) * a;
                }
            // X_C <- X_C L^-H, the same solve on every row of X_C (rows independent)
            for (int r = threadIdx.x; r < n; r += blockDim.x) {
                double2 row[RF_CMAX];
                for (int j = 0; j < m; ++j) {
                    double2 a = X[(int64_t)(c0 + j) * d.ld + r];
                    for (int k = 0; k < j; ++k) a = a - row[k] * conj(W[j + k * RF_CMAX]);
                    row[j] = (1.0 / W[j + j * RF_CMAX].x) * a;
                    X[(int64_t)(c0 + j) * d.ld + r] = row[j];
                }
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

// ================================================================== band G (first and hybrid second step)
// Both the first step and the second step below the size of a full one take C = X^H W for all
// pairs on the tensor cores but G = X^H X only on the band |i - j| <= RF_W: (lam0_j - lam_j) G_ij,
// the only place an entry off the band enters the update of a non-clustered pair, is negligible
// (|G_ij| ~ eps32 before the first step, of the size of its second-order error after it), and a
// cluster wider than the band meets G_ij ~ 0 outside it in the update; the cluster separation
// then forms the cluster's own Gram matrix from X.  Only near pairs need G to FP64 accuracy.
#define RF_BC 32            // columns per CTA
#define RF_BR 16            // rows per staged chunk

// G = X^H X on the band |i - j| <= RF_W in double-FP32, written into the full n x n G (column-major,
// ld); its other entries are left as they are (the update reads G only on the band then).
__global__ void __launch_bounds__(256) k_gram_band_df32(const MmfDesc* __restrict__ descs,
                                                        const int* __restrict__ idx,
                                                        const double2* __restrict__ Xg,
                                                        double2* __restrict__ Gg) {
    __shared__ Split xs[RF_BR][RF_BC + 2 * RF_W + 1];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    const int i0 = blockIdx.x * RF_BC;
    if (i0 >= n) return;
    const int cbase = i0 - RF_W;             // first staged column
    const int ncs = RF_BC + 2 * RF_W;         // staged columns
    const double2* X = Xg + d.mat_off;
    // each thread owns up to 5 (i, j) pairs: pair p = tid + 256 q, i = i0 + p / BW, j = i + p % BW - W
    DF gr[5], gi[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) gr[q] = gi[q] = DF{0.f, 0.f};
    for (int k0 = 0; k0 < n; k0 += RF_BR) {
        for (int e = threadIdx.x; e < RF_BR * ncs; e += 256) {
            const int c = e / RF_BR, kk = e - c * RF_BR;
            const int col = cbase + c, k = k0 + kk;
            const bool ok = k < n && col >= 0 && col < n;
            xs[kk][c] = split(ok ? X[(int64_t)col * d.ld + k] : make_double2(0.0, 0.0));
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 5; ++q) {
            const int p = threadIdx.x + 256 * q;
            if (p < RF_BC * RF_BW) {
                const int ii = p / RF_BW, off = p - ii * RF_BW;  // column i0+ii, partner i0+ii+off-W
                const int cix = ii + RF_W, cj = ii + off;           // staged indices
                for (int kk = 0; kk < RF_BR; ++kk) df_cmacc(gr[q], gi[q], xs[kk][cix], xs[kk][cj]);
                df_renorm(gr[q]); df_renorm(gi[q]);
            }
        }
        __syncthreads();
    }
    double2* G = Gg + d.mat_off;
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        const int p = threadIdx.x + 256 * q;
        if (p < RF_BC * RF_BW) {
            const int ii = p / RF_BW, off = p - ii * RF_BW;
            const int i = i0 + ii, j = i + off - RF_W;
            if (i < n && j >= 0 && j < n) {
                double2 g = make_double2((double)gr[q].hi + (double)gr[q].lo, (double)gi[q].hi + (double)gi[q].lo);
                if (i == j) g.y = 0.0;
                G[(int64_t)j * d.ld + i] = g;
            }
        }
    }
}


// The refinement is launched in parts so that the host can time the FP64-accurate Gram product
// on its own and choose the second step per system:
//   pre:    HX = H_F X, C = X^H W (and C' = X1^H Dx for a second full step) on the tensor cores
//   band_g: G on the band (first step, hybrid second step)
//   gram:   all of G = X1^H X1 in double-FP32 (+ C' + C'^H) for a full second step
//   update: lam, Et, X <- X + X Et, cluster separation;   finish: final ordering.
cudaError_t mmf_launch_refine_split_coef(const double2* coef, float4* cs, int64_t count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    k_split_coef<<<(int)std::min<int64_t>((count + 255) / 256, 1024), 256, 0, st>>>(coef, cs, count);
    return cudaGetLastError();
}

// HX = H_F X in double-FP32; X1 = fl32(X) is left in place for the Gram product.  Xlo: FP32
// remainder buffer (used only when X is not FP32-exact).
static void apply_hf(const MmfLaunch& L, const float4* cs, const int* pat, const double2* X, float2* X1, float2* Xlo,
                     double2* HX) {
    k_split_x<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, X1, Xlo);
    k_apply_hf_df32<<<dim3((L.nmax + 255) / 256, (L.nmax + 15) / 16, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, cs, pat, X1, Xlo, HX);
}

cudaError_t mmf_launch_coef_pattern(const MmfLaunch& L, const double2* coef, int* pat) {
    if (L.count <= 0) return cudaSuccess;
    k_coef_pattern<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, coef, pat);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_pre(const MmfLaunch& L, const float4* cs, const int* pat, const double2* X,
                                  const double* lam0, double2* HX, double2* T, float2* X1, void* ops, void* jobs,
                                  int* status, int second) {
    if (L.count <= 0) return cudaSuccess;
    // the first step's X holds FP32 eigenvectors (no remainder); the remainder of a second step's
    // X goes to T, which is free until C is written
    apply_hf(L, cs, pat, X, X1, second ? reinterpret_cast<float2*>(T) : nullptr, HX);
    k_w_prep_B<<<dim3(512, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, HX, lam0, ops);
    k_w_prep_A<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X1, ops);
    k_w_jobs<<<(L.count + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, L.count, ops, T, 0, (Tf3Job*)jobs);
    cudaError_t e = mmf_launch_tf3(jobs, L.count, L.nmax, 2 * L.nmax, status, L.stream);
    if (e != cudaSuccess || second != 1) return e;
    k_d_prep_B<<<dim3(512, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, ops);
    k_w_jobs<<<(L.count + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, L.count, ops, T, 1, (Tf3Job*)jobs);
    return mmf_launch_tf3(jobs, L.count, L.nmax, 2 * L.nmax, status, L.stream);
}

cudaError_t mmf_launch_refine_gram(const MmfLaunch& L, const float2* X1, double2* G, const double2* T, int second) {
    if (L.count <= 0) return cudaSuccess;
    const int nt = (L.nmax + RF_TILE - 1) / RF_TILE;
    // G of X1 = fl32(X) (written by the pre part): X itself in the first step (FP32
    // eigenvectors), its head in a second full step
    k_gram_x1<<<dim3(nt * (nt + 1) / 2, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X1, G);
    if (second) k_gram_fix<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, T);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_gram_fix(const MmfLaunch& L, double2* G, const double2* T) {
    if (L.count <= 0) return cudaSuccess;
    k_gram_fix<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, T);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_update(const MmfLaunch& L, const double2* coef, const int* pat, double2* X,
                                     const float2* X1,
                                     const double* lam0, double2* G, double2* HX, const double2* T, double* lam,
                                     int* status, int* cid, void* ops, void* jobs, double2* Eb,
                                     int band_fp32, int g_band) {
    if (L.count <= 0) return cudaSuccess;
    k_oa_lambda<<<L.count, 256, 0, L.stream>>>(L.desc, L.idx, G, T, lam0, lam, cid);
    k_oa_etilde<<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, T, lam0, lam, cid, g_band);
    // X <- X + X Et: band in double-FP32 (FP32 when another step follows), the rest on the tensor
    // cores (split TF32)
    k_et_band<<<dim3(64, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, Eb);
    k_xe_prep_B<<<dim3(512, L.count), 256, 0, L.stream>>>(L.desc, L.idx, G, ops);
    k_xe_prep_A<<<dim3(tf3_nq(L.nmax) * 4, (L.nmax + 31) / 32, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X1,
                                                                                             ops);
    k_xe_jobs<<<(L.count + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, L.count, ops, G, (Tf3Job*)jobs);
    cudaError_t e = mmf_launch_tf3(jobs, L.count, L.nmax, 2 * L.nmax, status, L.stream);
    if (e != cudaSuccess) return e;
    k_xe_apply<<<dim3((L.nmax + XT_R - 1) / XT_R, (L.nmax + XT_C - 1) / XT_C, L.count), 256, 0, L.stream>>>(
        L.desc, L.idx, X, X1, G, Eb, band_fp32);
    k_cluster_sep<<<dim3(std::min(L.nmax, 1024), L.count), 256, 0, L.stream>>>(L.desc, L.idx, coef, pat, X, HX, lam,
                                                                                cid, status);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_band_g(const MmfLaunch& L, const double2* X, double2* G) {
    if (L.count <= 0) return cudaSuccess;
    k_gram_band_df32<<<dim3((L.nmax + RF_BC - 1) / RF_BC, L.count), 256, 0, L.stream>>>(L.desc, L.idx, X, G);
    return cudaGetLastError();
}

cudaError_t mmf_launch_refine_finish(const MmfLaunch& L, double2* X, double* E, const double* lam, double2* S,
                                     int64_t mat_elems) {
    if (L.count <= 0) return cudaSuccess;
    k_sort_pairs<<<dim3(L.nmax, L.count), 256, 0, L.stream>>>(L.desc, L.idx, lam, X, E, S);
    cudaError_t e = cudaMemcpyAsync(X, S, sizeof(double2) * mat_elems, cudaMemcpyDeviceToDevice, L.stream);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}
