// k_bt_tc.cu -- S5 of the mixed path on the tensor cores: Z = Q Y, Q = P_0 P_1 ... P_{n-2}
// the Householder reflectors of the reduction (the eigenvectors of H_F from those of the
// tridiagonal matrix, Sec. 3.2's diagonalisation step).
//
// The reflectors are applied in super-blocks of MMF_BT_SB = 128, from the last to the first,
// each in compact WY form (Schreiber & Van Loan 1989): P_k0 ... P_{k0+127} = I - V T V^H, T upper
// triangular.  Only rows k0 .. n-1 of Z change; V vanishes on row k0, so that row range starts
// on an aligned row.  Per super-block:
//   G = V^H V                 T(c, c) = tau_c,  T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c)
//   P = Z^H V   (n x 128)     Q = P T^H   (n x 128)     Z <- Z - V Q^H
// G, P, Q and the update are real split-TF32 products on the tcgen05 engine (k_tf3_gemm): complex
// operands are stacked [Re | Im] along K, and each product's result goes straight into the tiled
// operand of the next one (P, Q) or is subtracted from Z.  The result has FP32 accuracy, as the
// SIMT back-transform's has; the refinement that follows takes the eigenvectors to FP64 accuracy.
#include <algorithm>

#include "mmf_internal.h"

// float offsets of one system's operands in its area (mmf_bt_floats(n) floats in all)
struct BtLayout {
    int64_t A1, B1, B3, AP, AQ, BT, G;
};
__host__ __device__ inline BtLayout bt_layout(int n) {
    const int K1 = 2 * mmf_bt_rp(n);
    BtLayout o;
    o.A1 = 0;                                     // Z^H stacked: n x K1
    o.B1 = o.A1 + 2 * tf3_piece(n, K1);           // V stacked: 256 x K1
    o.B3 = o.B1 + 2 * tf3_piece(256, K1);         // V by rows: 2R x 256
    o.AP = o.B3 + 2 * tf3_piece(2 * n, 256);      // P: n x 256
    o.AQ = o.AP + 2 * tf3_piece(n, 256);          // Q: n x 256
    o.BT = o.AQ + 2 * tf3_piece(n, 256);          // T stacked: 256 x 256
    o.G = o.BT + 2 * tf3_piece(256, 256);         // G = V^H V stacked, 256 x 256 row-major
    return o;
}

__device__ __forceinline__ float* bt_area(void* pool, const MmfDesc& d) {
    return reinterpret_cast<float*>(reinterpret_cast<uint16_t*>(pool) + d.oz_off);
}

// four consecutive K entries (k a multiple of 4) of row r, as TF32 pieces
__device__ __forceinline__ void bt_put4(float* P, int rows, int K, int r, int k, float4 v) {
    const float4 h = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z), tf32_round(v.w));
    const float4 l = make_float4(tf32_round(v.x - h.x), tf32_round(v.y - h.y), tf32_round(v.z - h.z),
                                 tf32_round(v.w - h.w));
    *reinterpret_cast<float4*>(P + tf3_pos(rows, K, 0, r, k)) = h;
    *reinterpret_cast<float4*>(P + tf3_pos(rows, K, 1, r, k)) = l;
}

__device__ __forceinline__ float4 neg4(float4 v) { return make_float4(-v.x, -v.y, -v.z, -v.w); }

// v_p[k0 + r] of reflector k0 + p: 0 for r <= p, 1 for r = p + 1, the stored entry below
__device__ __forceinline__ float2 bt_refl(const float2* __restrict__ A, int ld, int k0, int p, int r, int R, int nbk) {
    if (p >= nbk || r >= R || r <= p) return make_float2(0.f, 0.f);
    if (r == p + 1) return make_float2(1.f, 0.f);
    return A[(k0 + r) + (int64_t)(k0 + p) * ld];
}

struct BtStep {
    int k0, R, Rp, K1, nbk;
};
// super-block handled by a system at step q (the last one at q = 0); false once it has none left
__device__ __forceinline__ bool bt_step(int n, int q, BtStep& s) {
    const int sb = mmf_bt_nsb(n) - 1 - q;
    if (sb < 0) return false;
    s.k0 = sb * MMF_BT_SB;
    s.R = n - s.k0;
    s.Rp = mmf_bt_rp(s.R);
    s.K1 = 2 * s.Rp;
    s.nbk = min(MMF_BT_SB, n - 1 - s.k0);
    return true;
}

// Z = Y (FP64 row-major n x n) as FP32 complex, column-major; 32 x 32 tiles through shared memory
__global__ void __launch_bounds__(256) k_bt_init(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                 const double* __restrict__ Yg, float2* __restrict__ Zg) {
    __shared__ float tile[32][33];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    if (r0 >= n || c0 >= n) return;
    const double* Y = Yg + d.sq_off;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int i = ty; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + tx;
        tile[i][tx] = (r < n && c < n) ? (float)Y[(int64_t)r * n + c] : 0.f;
    }
    __syncthreads();
    float2* Z = Zg + d.mat_off;
    for (int i = ty; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + tx;
        if (r < n && c < n) Z[r + (int64_t)c * d.ld] = make_float2(tile[tx][i], 0.f);
    }
}

// Operands of step q: A1 = Z^H stacked (row c: [Re Z(k0.., c) | Im Z(k0.., c)], halves Rp long),
// B1 = V stacked (rows p: [Re v_p | Im v_p], rows 128 + p: [Im v_p | -Re v_p]),
// B3 = V by rows (rows 2r: [Re V(r, :) | Im V(r, :)], rows 2r + 1: [Im V(r, :) | -Re V(r, :)]).
// Padding rows and K entries are written as zeros.
__global__ void __launch_bounds__(256) k_bt_prep(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                 void* pool, const float2* __restrict__ H,
                                                 const float2* __restrict__ Zg, int q) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, ld = d.ld;
    BtStep s;
    if (!bt_step(n, q, s)) return;
    float* W = bt_area(pool, d);
    const BtLayout o = bt_layout(n);
    const float2* A = H + d.mat_off;
    const float2* Z = Zg + d.mat_off + s.k0;
    const int rc = s.Rp / 4;                          // 4-row chunks per half
    const int64_t nA1 = (int64_t)tf3_nq(n) * 128 * rc;
    const int64_t nB1 = (int64_t)MMF_BT_SB * rc;
    const int half3 = tf3_nq(2 * s.R) * 64;           // row pairs of B3, padding included
    const int64_t nB3 = (int64_t)half3 * (MMF_BT_SB / 4);
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nA1 + nB1 + nB3;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nA1) {
            const int c = (int)(e / rc), r = 4 * (int)(e - (int64_t)c * rc);
            float4 re = z4, im = z4;
            if (c < n) {
                const float2* zc = Z + (int64_t)c * ld + r;   // 32-byte aligned: k0, r, ld multiples of 4
                if (r + 3 < s.R) {
                    const float4 a = reinterpret_cast<const float4*>(zc)[0], b = reinterpret_cast<const float4*>(zc)[1];
                    re = make_float4(a.x, a.z, b.x, b.z);
                    im = make_float4(a.y, a.w, b.y, b.w);
                } else {
                    float rv[4], iv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float2 z = (r + u < s.R) ? zc[u] : make_float2(0.f, 0.f);
                        rv[u] = z.x;
                        iv[u] = z.y;
                    }
                    re = make_float4(rv[0], rv[1], rv[2], rv[3]);
                    im = make_float4(iv[0], iv[1], iv[2], iv[3]);
                }
            }
            bt_put4(W + o.A1, n, s.K1, c, r, re);
            bt_put4(W + o.A1, n, s.K1, c, s.Rp + r, im);
        } else if (e < nA1 + nB1) {
            const int64_t f = e - nA1;
            const int p = (int)(f / rc), r = 4 * (int)(f - (int64_t)p * rc);
            float rv[4], iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 v = bt_refl(A, ld, s.k0, p, r + u, s.R, s.nbk);
                rv[u] = v.x;
                iv[u] = v.y;
            }
            const float4 vr = make_float4(rv[0], rv[1], rv[2], rv[3]), vi = make_float4(iv[0], iv[1], iv[2], iv[3]);
            bt_put4(W + o.B1, 256, s.K1, p, r, vr);
            bt_put4(W + o.B1, 256, s.K1, p, s.Rp + r, vi);
            bt_put4(W + o.B1, 256, s.K1, MMF_BT_SB + p, r, vi);
            bt_put4(W + o.B1, 256, s.K1, MMF_BT_SB + p, s.Rp + r, neg4(vr));
        } else {
            const int64_t f = e - nA1 - nB1;
            const int pc = (int)(f / half3), r = (int)(f - (int64_t)pc * half3);
            const int p = 4 * pc;
            float rv[4], iv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float2 v = bt_refl(A, ld, s.k0, p + u, r, s.R, s.nbk);
                rv[u] = v.x;
                iv[u] = v.y;
            }
            const float4 vr = make_float4(rv[0], rv[1], rv[2], rv[3]), vi = make_float4(iv[0], iv[1], iv[2], iv[3]);
            bt_put4(W + o.B3, 2 * s.R, 256, 2 * r, p, vr);
            bt_put4(W + o.B3, 2 * s.R, 256, 2 * r, MMF_BT_SB + p, vi);
            bt_put4(W + o.B3, 2 * s.R, 256, 2 * r + 1, p, vi);
            bt_put4(W + o.B3, 2 * s.R, 256, 2 * r + 1, MMF_BT_SB + p, neg4(vr));
        }
    }
}

// The four products of step q for every system (M = 0 where the system has no super-block left):
//   0: G = B1 B1^T (row-major 256 x 256)   1: P = A1 B1^T -> AP   2: Q = AP BT^T -> AQ
//   3: Z(k0.., :) -= (AQ B3^T) as the rows of Z^H (interleaved Re, Im)
__global__ void k_bt_jobs(const MmfDesc* __restrict__ descs, const int* __restrict__ idx, int count, void* pool,
                          float2* Zg, int q, Tf3Job* jobs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const MmfDesc d = descs[idx[i]];
    const int n = d.n;
    BtStep s;
    const bool on = bt_step(n, q, s);
    float* W = bt_area(pool, d);
    const BtLayout o = bt_layout(n);
    Tf3Job j[4];
    j[0].A = W + o.B1; j[0].B = W + o.B1; j[0].C = W + o.G;
    j[0].M = 256; j[0].N = 256; j[0].K = on ? s.K1 : 32; j[0].ldc = 256; j[0].mode = TF3_STORE;
    j[1].A = W + o.A1; j[1].B = W + o.B1; j[1].C = W + o.AP;
    j[1].M = n; j[1].N = 256; j[1].K = on ? s.K1 : 32; j[1].ldc = 0; j[1].mode = TF3_OPERAND;
    j[2].A = W + o.AP; j[2].B = W + o.BT; j[2].C = W + o.AQ;
    j[2].M = n; j[2].N = 256; j[2].K = 256; j[2].ldc = 0; j[2].mode = TF3_OPERAND;
    j[3].A = W + o.AQ; j[3].B = W + o.B3; j[3].C = reinterpret_cast<float*>(Zg + d.mat_off + (on ? s.k0 : 0));
    j[3].M = n; j[3].N = on ? 2 * s.R : 0; j[3].K = 256; j[3].ldc = 2 * d.ld; j[3].mode = TF3_SUBTRACT;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        if (!on) j[g].M = 0;
        jobs[(int64_t)g * count + i] = j[g];
    }
}

// T of step q from G (strict upper triangle), written stacked as BT (rows p: [Re T(p, :) |
// Im T(p, :)], rows 128 + p: [-Im T(p, :) | Re T(p, :)]).  One CTA per system; S[i][j] holds T(i, j)
// for j >= i and G(j, i) for j < i.
#define BT_TF_THREADS 512
#define BT_SS (MMF_BT_SB + 1)
__global__ void __launch_bounds__(BT_TF_THREADS) k_bt_tfac(const MmfDesc* __restrict__ descs,
                                                           const int* __restrict__ idx, void* pool,
                                                           const float2* __restrict__ taup, int q) {
    extern __shared__ float2 S[];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n;
    BtStep s;
    if (!bt_step(n, q, s)) return;
    float* W = bt_area(pool, d);
    const BtLayout o = bt_layout(n);
    const float* G = W + o.G;
    const float2* tau = taup + d.vec_off;
    const int tid = threadIdx.x;
    for (int e = tid; e < MMF_BT_SB * MMF_BT_SB; e += BT_TF_THREADS) {
        const int a = e % MMF_BT_SB, b = e / MMF_BT_SB;   // S[a][b]
        S[a * BT_SS + b] = (b >= a) ? make_float2(0.f, 0.f)
                                    : make_float2(G[b * 256 + a], G[b * 256 + MMF_BT_SB + a]);  // G(b, a)
    }
    __syncthreads();
    for (int c = 0; c < s.nbk; ++c) {
        const float2 tc = tau[s.k0 + c];
        if (tid < c) {
            float2 acc = make_float2(0.f, 0.f);
            for (int k = tid; k < c; ++k) acc = acc + S[tid * BT_SS + k] * S[c * BT_SS + k];
            S[tid * BT_SS + c] = make_float2(-(tc.x * acc.x - tc.y * acc.y), -(tc.x * acc.y + tc.y * acc.x));
        }
        if (tid == 0) S[c * BT_SS + c] = tc;
        __syncthreads();
    }
    for (int e = tid; e < MMF_BT_SB * (MMF_BT_SB / 4); e += BT_TF_THREADS) {
        const int p = e / (MMF_BT_SB / 4), k = 4 * (e % (MMF_BT_SB / 4));
        float tr[4], ti[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float2 t = (k + u >= p) ? S[p * BT_SS + k + u] : make_float2(0.f, 0.f);
            tr[u] = t.x;
            ti[u] = t.y;
        }
        const float4 r4 = make_float4(tr[0], tr[1], tr[2], tr[3]), i4 = make_float4(ti[0], ti[1], ti[2], ti[3]);
        bt_put4(W + o.BT, 256, 256, p, k, r4);
        bt_put4(W + o.BT, 256, 256, p, MMF_BT_SB + k, i4);
        bt_put4(W + o.BT, 256, 256, MMF_BT_SB + p, k, neg4(i4));
        bt_put4(W + o.BT, 256, 256, MMF_BT_SB + p, MMF_BT_SB + k, r4);
    }
}

// hn: host copy of n for each system of the launch; jobs: 4 x count Tf3Job; *launches gets the
// number of kernels launched
cudaError_t mmf_launch_backtransform_tc(const MmfLaunch& L, const int* hn, const void* H, const void* tau,
                                        const double* Y, void* Z, void* pool, void* jobs, int* err,
                                        int* launches) {
    *launches = 0;
    if (L.count <= 0) return cudaSuccess;
    int maxnsb = 0;
    for (int i = 0; i < L.count; ++i) maxnsb = std::max(maxnsb, mmf_bt_nsb(hn[i]));
    const int nb = (L.nmax + 31) / 32;
    k_bt_init<<<dim3(nb, nb, L.count), 256, 0, L.stream>>>(L.desc, L.idx, Y, (float2*)Z);
    const size_t smt = sizeof(float2) * MMF_BT_SB * BT_SS;
    cudaError_t e = cudaFuncSetAttribute(k_bt_tfac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smt);
    if (e != cudaSuccess) return e;
    Tf3Job* J = (Tf3Job*)jobs;
    int nl = 1;
    for (int q = 0; q < maxnsb; ++q) {
        int N3 = 0;
        int64_t items = 0;
        for (int i = 0; i < L.count; ++i) {
            const int n = hn[i], sb = mmf_bt_nsb(n) - 1 - q;
            if (sb < 0) continue;
            const int R = n - sb * MMF_BT_SB, rc = mmf_bt_rp(R) / 4;
            N3 = std::max(N3, 2 * R);
            items = std::max<int64_t>(items, (int64_t)tf3_nq(n) * 128 * rc + (int64_t)MMF_BT_SB * rc +
                                                 (int64_t)tf3_nq(2 * R) * 64 * (MMF_BT_SB / 4));
        }
        const int gx = (int)std::min<int64_t>((items + 255) / 256, 1024);
        k_bt_jobs<<<(L.count + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, L.count, pool, (float2*)Z, q, J);
        k_bt_prep<<<dim3(gx, L.count), 256, 0, L.stream>>>(L.desc, L.idx, pool, (const float2*)H, (const float2*)Z, q);
        if ((e = mmf_launch_tf3(J, L.count, 256, 256, err, L.stream)) != cudaSuccess) return e;
        k_bt_tfac<<<dim3(1, L.count), BT_TF_THREADS, smt, L.stream>>>(L.desc, L.idx, pool, (const float2*)tau, q);
        if ((e = mmf_launch_tf3(J + L.count, L.count, L.nmax, 256, err, L.stream)) != cudaSuccess) return e;
        if ((e = mmf_launch_tf3(J + 2 * L.count, L.count, L.nmax, 256, err, L.stream)) != cudaSuccess) return e;
        if ((e = mmf_launch_tf3(J + 3 * L.count, L.count, L.nmax, N3, err, L.stream)) != cudaSuccess) return e;
        nl += 7;
    }
    *launches = nl;
    return cudaGetLastError();
}
