// mmf_internal.h -- device-side data layout and helpers shared by the CUDA kernels.
//
// One "batch" holds many independent driven systems (Eq. 1).  Each system has a
// descriptor with its sizes and the offsets of its slices in the batch's device pools.
// All n x n matrices are column-major with leading dimension ld (a multiple of 4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MMF_MAX_MODES 4

struct MmfDesc {
    int32_t D, K, M, n;                 // levels, modes, Fourier blocks, n = D * M
    int32_t ld, b0, small, pat_cap;     // leading dim, central block index, Jacobi flag,
                                        // nonzeros kept per coefficient row (0: dense rows)
    int32_t band, pad0;                 // half-bandwidth when reduced by the bulge chase (0: dense)
    int32_t N[MMF_MAX_MODES];           // truncation |n_k| <= N_k
    int32_t nharm[MMF_MAX_MODES];       // harmonics per mode (couplings V^{k,1..nharm})
    int32_t S[MMF_MAX_MODES];           // block strides, S_0 = 1, S_k = prod_{k'<k}(2N_k'+1)
    double omega[MMF_MAX_MODES];
    int64_t coef_off;   // double2 offset of H0 (D x D row-major); V^{k,h} follow (mode, harmonic)
    int64_t mat_off;    // element offset of this system's n x ld matrices in matrix pools
    int64_t vec_off;    // element offset of its length-n vectors (packed)
    int64_t sq_off;     // element offset of its n x n row-major scratch (tridiagonal solver)
    int64_t pan_off;    // element offset of its n x NB panels (Householder) / T factors
    int64_t t_off;      // offset of its nt times
    int64_t f_off;      // double2 offset of its nt x M Fourier phase table
    int64_t u_off;      // double2 offset of its nt x D x D time-evolution output
    int64_t p_off;      // offset of its D x D transition-probability output
    int64_t oz_off;     // BF16 offset of its Gram-product slices (mixed path)
    int64_t pat_off;    // int offset of its coefficient nonzero pattern (mixed path)
};

// Nonzero pattern of a system's coefficient rows (refinement's H_F products), rebuilt on the
// device from the current coefficients before every refinement.  Matrices m = 0 (H0 rows),
// then per coupling q (mode-major, harmonic-minor) m = 1 + 2q (rows of V) and m = 2 + 2q (rows
// of V^dagger, i.e. columns of V).  Layout at pat + pat_off: [0] = 1 when every row has at most
// pat_cap nonzeros (else the kernels take the dense rows), then nm D counts, then nm D pat_cap
// column indices.
__host__ __device__ __forceinline__ int coef_matrices(const MmfDesc& d) {
    int nm = 1;
    for (int l = 0; l < d.K; ++l) nm += 2 * d.nharm[l];
    return nm;
}

// ------------------------------------------------------------------ complex helpers
template <class R> struct Cx;
template <> struct Cx<double> { typedef double2 T; };
template <> struct Cx<float> { typedef float2 T; };

__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }

template <class C> __device__ __forceinline__ C czero();
template <> __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }

#define MMF_CX_OPS(C, R)                                                                      \
    __device__ __forceinline__ C operator+(C a, C b) { return mk(a.x + b.x, a.y + b.y); }     \
    __device__ __forceinline__ C operator-(C a, C b) { return mk(a.x - b.x, a.y - b.y); }     \
    __device__ __forceinline__ C operator*(C a, C b) {                                       \
        return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);                             \
    }                                                                                         \
    __device__ __forceinline__ C operator*(R s, C a) { return mk(s * a.x, s * a.y); }        \
    __device__ __forceinline__ C conj(C a) { return mk(a.x, -a.y); }                         \
    /* conj(a) * b */                                                                         \
    __device__ __forceinline__ C cmulc(C a, C b) {                                           \
        return mk(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);                             \
    }                                                                                         \
    __device__ __forceinline__ R abs2(C a) { return a.x * a.x + a.y * a.y; }

MMF_CX_OPS(double2, double)
MMF_CX_OPS(float2, float)

__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2(a.x, a.y); }
template <class C> __device__ __forceinline__ C from_c128(double2 a);
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 a) { return a; }
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 a) {
    return make_float2(__double2float_rn(a.x), __double2float_rn(a.y));
}

template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Fourier vector of block b: n_k = (b / S_k) mod (2N_k+1) - N_k
__device__ __forceinline__ void block_nvec(const MmfDesc& d, int b, int* nv) {
#pragma unroll
    for (int k = 0; k < MMF_MAX_MODES; ++k) {
        if (k < d.K) {
            int w = 2 * d.N[k] + 1;
            nv[k] = (b / d.S[k]) % w - d.N[k];
        } else {
            nv[k] = 0;
        }
    }
}

// n.omega accumulated over k ascending, each product and sum rounded once (no FMA)
__device__ __forceinline__ double block_ndotw(const MmfDesc& d, int b) {
    int nv[MMF_MAX_MODES];
    block_nvec(d, b, nv);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < MMF_MAX_MODES; ++k)
        if (k < d.K) s = __dadd_rn(s, __dmul_rn((double)nv[k], d.omega[k]));
    return s;
}

// Double-FP32 arithmetic: FP64-accurate sums of products computed on the FP32 pipes.
// Every FP64 value is split x = x1 + x2 (x1 = fl32(x), x2 = fl32(x - x1)); x1*y1 is taken exactly
// (product + FMA error term), the cross terms in FP32, and sums are accumulated as a (hi, lo)
// pair with TwoSum (Knuth 1969).
struct DF {
    float hi, lo;
};

// acc += a * b with a = a1 + a2, b = b1 + b2 (FP32 pieces of FP64 values)
__device__ __forceinline__ void df_mac(DF& acc, float a1, float a2, float b1, float b2) {
    const float p = a1 * b1;
    const float e = fmaf(a1, b1, -p);
    const float c = fmaf(a1, b2, a2 * b1);
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += err + e + c;
}
// acc += a1 * (b1 + b2) with a1 exactly FP32 (no a2 piece)
__device__ __forceinline__ void df_mac1(DF& acc, float a1, float b1, float b2) {
    const float p = a1 * b1;
    const float e = fmaf(a1, b1, -p);
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += err + fmaf(a1, b2, e);
}
// acc += a1 * b1 with both exactly FP32
__device__ __forceinline__ void df_mac11(DF& acc, float a1, float b1) {
    const float p = a1 * b1;
    const float e = fmaf(a1, b1, -p);
    const float s = acc.hi + p;
    const float bb = s - acc.hi;
    const float err = (acc.hi - (s - bb)) + (p - bb);
    acc.hi = s;
    acc.lo += err + e;
}
__device__ __forceinline__ void df_renorm(DF& a) {
    const float s = a.hi + a.lo;
    a.lo = a.lo - (s - a.hi);
    a.hi = s;
}

struct Split {  // FP32 pieces of one complex FP64 value
    float r1, r2, i1, i2;
};
__device__ __forceinline__ Split split(double2 v) {
    Split s;
    s.r1 = __double2float_rn(v.x);
    s.r2 = __double2float_rn(v.x - (double)s.r1);
    s.i1 = __double2float_rn(v.y);
    s.i2 = __double2float_rn(v.y - (double)s.i1);
    return s;
}

// conj(a) * b accumulated into (re, im)
__device__ __forceinline__ void df_cmacc(DF& re, DF& im, const Split& a, const Split& b) {
    df_mac(re, a.r1, a.r2, b.r1, b.r2);
    df_mac(re, a.i1, a.i2, b.i1, b.i2);
    df_mac(im, a.r1, a.r2, b.i1, b.i2);
    df_mac(im, -a.i1, -a.i2, b.r1, b.r2);
}

// a * b accumulated into (re, im)
__device__ __forceinline__ void df_cmac(DF& re, DF& im, const Split& a, const Split& b) {
    df_mac(re, a.r1, a.r2, b.r1, b.r2);
    df_mac(re, -a.i1, -a.i2, b.i1, b.i2);
    df_mac(im, a.r1, a.r2, b.i1, b.i2);
    df_mac(im, a.i1, a.i2, b.r1, b.r2);
}
__device__ __forceinline__ double2 df_value(const DF& re, const DF& im) {
    return make_double2((double)re.hi + (double)re.lo, (double)im.hi + (double)im.lo);
}


// ------------------------------------------------------------------ status codes (device)
#define MMF_ST_OK 0
#define MMF_ST_NOCONV 1      // iteration cap reached
#define MMF_ST_NONFINITE 2   // NaN / Inf encountered
#define MMF_ST_CLUSTER 3     // refinement cluster too large to separate

// ------------------------------------------------------------------ kernel launchers
// Every launcher takes the device descriptor array and a device list of system indices.
// ------------------------------------------------------------------ band path: reflector store
// Pass s of the bulge chase holds the reflectors of sweeps j = 0 .. n-2-s b (n-1-s b of them)
// starting at off(s) = s (n-1) - b s (s-1) / 2.  Reflector (j, s): v at V[(off(s) + j) b + i],
// i < b (zero beyond its length), tau at T[off(s) + j] with T = V + nref b; it acts on rows
// j + 1 + s b .. j + s b + b.
__host__ __device__ __forceinline__ int64_t sbr_off(int n, int b, int s) {
    return (int64_t)s * (n - 1) - (int64_t)b * s * (s - 1) / 2;
}
__host__ __device__ __forceinline__ int sbr_passes(int n, int b) { return (n - 2) / b + 1; }
__host__ __device__ __forceinline__ int64_t sbr_nref(int n, int b) { return sbr_off(n, b, sbr_passes(n, b)); }
// Row-major Z of the band back-transform in the system's inverse-iteration work slot (3 n^2
// doubles from work + 3 sq_off, free after the tridiagonal solve): from the slot's first 16-byte
// boundary (the slot starts 8-byte aligned; Z needs at most 2 n^2 doubles plus 8 bytes).
__device__ __forceinline__ void* sbr_zbase(double* work, const MmfDesc& d) {
    const uintptr_t p = (uintptr_t)(work + 3 * d.sq_off);
    return (void*)((p + 15) & ~(uintptr_t)15);
}

struct MmfLaunch {
    const MmfDesc* desc;     // device
    const int* idx;          // device: systems in this launch
    int count;               // number of systems in this launch
    int nmax;                // largest n among them
    cudaStream_t stream;
};

cudaError_t mmf_launch_assemble(const MmfLaunch& L, const double2* coef, void* H, int fp32);
cudaError_t mmf_launch_jacobi(const MmfLaunch& L, void* H, void* Zw, double* E, void* Z,
                              int* status, int fp32, int max_sweeps);
// tc (FP32 only): the trailing update of each panel on the tensor cores in split TF32; status:
// per-system status words (a tensor-core wait that gave up sets MMF_ST_NOCONV)
cudaError_t mmf_launch_hetrd(const MmfLaunch& L, void* H, void* Vp, void* Wp, double* dvec,
                             double* evec, void* tau, int fp32, int tc, int* status);
cudaError_t mmf_launch_tridiag_eig(const MmfLaunch& L, const double* dvec, const double* evec,
                                   double* aux, double* e2, double* E, double* Y, double* work,
                                   int* status, int fp32, int iters);
cudaError_t mmf_launch_backtransform(const MmfLaunch& L, const void* H, const void* tau,
                                     void* Tf, const double* Y, void* Z, int fp32);
cudaError_t mmf_launch_widen(const MmfLaunch& L, const void* Zp, double2* Z, int fp32);
cudaError_t mmf_launch_outputs(const MmfLaunch& L, int Mmax, int Dmax, const double* E,
                               const double2* Z, float2* Z1, float2* Zlo, const double* t, double t0, int nt,
                               double2* F, double2* U, double* P, double cluster_rel, int skip_u,
                               void* scratch, int scratch_esz);
int mmf_hetrd_max_n(int fp32);
// banded H_F (k_sbr.cu): bulge chase to real tridiagonal form (d, e; reflectors kept in the
// system's FP64 eigenvector slot), then Z = Q Y into the back-transform's output (Zp)
int mmf_sbr_class(int band);                 // window class 8/16/32/64, 0 if the band is wider
int64_t mmf_sbr_store_elems(int n, int band);  // complex elements of the reflector store
cudaError_t mmf_launch_sbr_chase(const MmfLaunch& L, int bmax, void* H, double2* store, double* dvec, double* evec,
                                 int* status, int fp32);
cudaError_t mmf_launch_sbr_bt(const MmfLaunch& L, int bmax, const double2* store, const double* Y, double* work,
                              void* Zout, int fp32);
// Z (row-major FP32, work slot) -> column-major FP32 output (mixed path)
cudaError_t mmf_launch_sbr_out(const MmfLaunch& L, double* work, float2* Zout);
// Band back-transform on the tensor cores (mixed path, half-bandwidth 33..64): per block of 64
// sweeps its compact-WY factors and both products' B operands into the system's operand area
// (pool + oz_off BF16 units, mmf_sbt_ops_elems), then one CTA per (system, 128 columns of Z)
// applying the blocks as split-TF32 products, then the transpose to Zout.  A tensor-core wait that
// gives up sets the system's status word to MMF_ST_NOCONV.
cudaError_t mmf_launch_sbr_bt_tc(const MmfLaunch& L, const double2* store, const double* Y, double* work, void* pool,
                                 float2* Zout, int* status);
int64_t mmf_sbt_ops_elems(int n, int b);  // operand-area size (BF16 units) of a system's blocks
// dressed basis (k_dressed.cu): zone representatives of the dressing batch, U_F at t1 and the
// full batch's times, and Ud = U_F(t2)^dagger U(t2, t1) U_F(t1) per time
cudaError_t mmf_launch_dressed(const MmfDesc* ddesc, const MmfDesc* fdesc, int count, int nmax_d, int Dmax,
                               const double2* Zd, const double* Ed, const double2* U, const double* t, double t1,
                               int nt, const int64_t* roff, const int64_t* ufoff, int64_t* reps, double* Ebar,
                               double2* UF, double2* Wt, double2* Ud, cudaStream_t st);
cudaError_t mmf_launch_hetrd_large(const MmfDesc& d, void* H, void* Vp, void* Wp, double* dvec, double* evec,
                                   void* tau, void* work, void* sc, int fp32, cudaStream_t st);
cudaError_t mmf_launch_micromotion(const MmfLaunch& L, int D, const double2* Z, const double* t,
                                   int nt, int64_t* reps, double2* UF);
cudaError_t mmf_launch_refine_split_coef(const double2* coef, float4* cs, int64_t count, cudaStream_t st);
cudaError_t mmf_launch_coef_pattern(const MmfLaunch& L, const double2* coef, int* pat);
cudaError_t mmf_launch_refine_pre(const MmfLaunch& L, const float4* cs, const int* pat, const double2* X, const double* lam0,
                                  double2* HX, double2* T, float2* X1, void* ops, void* jobs, int* status,
                                  int second);
cudaError_t mmf_launch_refine_gram(const MmfLaunch& L, const float2* X1, double2* G, const double2* T, int second);
cudaError_t mmf_launch_refine_gram_fix(const MmfLaunch& L, double2* G, const double2* T);
// one Ogita-Aishima update (lam, Et, X <- X + X Et in place, cluster separation).  band_fp32: apply
// the near band of Et in FP32 (only when another full-accuracy step follows); g_band: G was formed
// only on the band |i - j| <= 16 and is taken as 0 off it.
cudaError_t mmf_launch_refine_update(const MmfLaunch& L, const double2* coef, const int* pat, double2* X, const float2* X1,
                                     const double* lam0, double2* G, double2* HX, const double2* T, double* lam,
                                     int* status, int* cid, void* ops, void* jobs, double2* Eb,
                                     int band_fp32, int g_band);
// first step and hybrid second step: G = X^H X on the band |i - j| <= 16 (double-FP32), the rest
// of G left unset (the update then runs with g_band = 1)
cudaError_t mmf_launch_refine_band_g(const MmfLaunch& L, const double2* X, double2* G);
cudaError_t mmf_launch_refine_finish(const MmfLaunch& L, double2* X, double* E, const double* lam, double2* S,
                                     int64_t mat_elems);
// Gram product on the BF16 tensor cores by exact integer slicing (k_ozaki.cu)
#define OZ_S 5
size_t mmf_ozaki_slice_elems(int n);
cudaError_t mmf_launch_ozaki_gram(const MmfLaunch& L, const float2* X1, void* S, int* exps, double2* G, int* err);
int mmf_ozaki_max_n();  // largest n the exact-slicing Gram product takes (int64 range)
// time evolution on the tensor cores (mixed path): Phi by exact slicing, then U in FP64; operands
// and Phi in the system's operand area (mmf_phi_elems BF16 units); Dmax <= mmf_phi_max_levels()
int64_t mmf_phi_elems(int n, int D, int M, int nt);
int mmf_phi_max_levels();
cudaError_t mmf_launch_phi(const MmfLaunch& L, int Dmax, int nt, const float2* Z1, const float2* Zlo,
                           const void* F, const double* E, const double2* Z, const double* t, double t0, void* pool,
                           double2* U, int* err);
int mmf_ozaki_selftest_impl(int n, double* max_abs, double* max_ref);
#define MMF_REFINE_BW 33   // entries per row of the refinement's band buffer (2 W + 1)
#define MMF_REFINE_FULL2_N 3000   // from this n on the second refinement step is a full one
// batched tensor-core GEMM (k_umma.cu): C(m, n) = sum_p sum_k A_p(m, k) B_p(n, k), K-major
// operands (TF32 in FP32 storage, or BF16), FP32 result
#define UM_MAXP 3
struct UmmaJob {
    const void* A[UM_MAXP];   // A_p: M x K, row stride lda elements (lda * element size % 16 == 0)
    const void* B[UM_MAXP];   // B_p: N x K, row stride ldb elements
    float* C;                 // M x N, row stride ldc
    int M, N, K;
    int lda, ldb, ldc;
};
cudaError_t mmf_launch_umma(const void* jobs, int count, int P, int Mmax, int Nmax, int kind, int* err,
                            cudaStream_t stream);

// Split-TF32 products on the tensor cores with pre-tiled operands (k_umma.cu, k_tf3_gemm):
//   C(m, n) = A1 B1^T + A1 B2^T + A2 B1^T   (A = A1 + A2, B = B1 + B2 in TF32 pieces)
// Each operand (rows x K) is stored as two pieces (A1 then A2), each in 128-row x 32-K tiles of
// 16 KB in the tensor cores' shared-memory layout (128-byte swizzle, K-major); tile (t, q) of a
// piece sits at ((t * nq + q) * 4096) floats, nq = ceil(rows / 128).  Padding rows and K columns
// hold zeros.
__host__ __device__ __forceinline__ int tf3_nq(int rows) { return (rows + 127) / 128; }
__host__ __device__ __forceinline__ int tf3_nt(int K) { return (K + 31) / 32; }
__host__ __device__ __forceinline__ int64_t tf3_piece(int rows, int K) {
    return (int64_t)tf3_nt(K) * tf3_nq(rows) * 4096;
}
__host__ __device__ __forceinline__ int64_t tf3_pos(int rows, int K, int piece, int r, int k) {
    const int t = k >> 5, kk = k & 31, q = r >> 7, rr = r & 127;
    return (((int64_t)piece * tf3_nt(K) + t) * tf3_nq(rows) + q) * 4096 + (rr >> 3) * 256 + (rr & 7) * 32 +
           (((kk >> 2) ^ (rr & 7)) << 2) + (kk & 3);
}
// Output modes: 0 stores C (M x N, row stride ldc); 1 subtracts the product from C; 2 writes the
// product's TF32 pieces as an operand of a further product (rows = M, K = N, a multiple of 32,
// piece 1 at C, piece 2 after tf3_piece(M, N) floats; padding rows written as zeros).
#define TF3_STORE 0
#define TF3_SUBTRACT 1
#define TF3_OPERAND 2
struct Tf3Job {
    const float* A;   // piece 1 of A (piece 2 follows after tf3_piece(M, K) floats)
    const float* B;   // piece 1 of B
    float* C;         // M x N, row stride ldc
    int M, N, K, ldc;
    int mode;
};
#ifdef __CUDACC__
// TF32 operands for the tcgen05 engine: round to nearest (ties away) to 10 explicit bits
__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}
#endif
cudaError_t mmf_launch_tf3(const void* jobs, int count, int Mmax, int Nmax, int* err, cudaStream_t stream);
// floats of the refinement's split-TF32 operands for one system (A: n x 2n, B: 2n x 2n)
__host__ __device__ __forceinline__ int64_t mmf_tf3_floats(int n) {
    return 2 * tf3_piece(n, 2 * n) + 2 * tf3_piece(2 * n, 2 * n);
}
int mmf_umma_selftest_impl(int M, int N, int K, int kind, int P, double* max_abs, double* max_ref);
int mmf_tf3_selftest_impl(int M, int N, int K, int mode, double* max_rel, double* max_rel_fp32);
int mmf_hetrd_selftest_impl(int n, int count, int tc, double* max_err, double* max_ref);

// Back-transform of the mixed path on the tensor cores (k_bt_tc.cu): reflectors in super-blocks
// of MMF_BT_SB, each applied as split-TF32 products.  Systems with n >= MMF_BT_TC_NMIN take it.
#define MMF_BT_SB 128
#define MMF_BT_TC_NMIN 256
__host__ __device__ __forceinline__ int mmf_bt_rp(int n) { return (n + 31) & ~31; }
__host__ __device__ __forceinline__ int mmf_bt_nsb(int n) { return (n - 1 + MMF_BT_SB - 1) / MMF_BT_SB; }
// floats of one system's back-transform operands (they live in the refinement's operand area)
cudaError_t mmf_launch_backtransform_tc(const MmfLaunch& L, const int* hn, const void* H, const void* tau,
                                        const double* Y, void* Z, void* pool, void* jobs, int* err,
                                        int* launches);
__host__ __device__ __forceinline__ int64_t mmf_bt_floats(int n) {
    const int K1 = 2 * mmf_bt_rp(n);
    return 2 * tf3_piece(n, K1) + 2 * tf3_piece(256, K1) + 2 * tf3_piece(2 * n, 256) + 4 * tf3_piece(n, 256) +
           2 * tf3_piece(256, 256) + 256 * 256;
}
#define MMF_MIN_LD 36   // n x ld matrix slots also hold the n x 33 band of the refinement

#define MMF_NB 32          // Householder panel width and back-transform block size
#define MMF_JACOBI_NMAX_F64 84
#define MMF_JACOBI_NMAX_F32 118
