// k_backtransform.cu -- S5: eigenvectors of H_F from those of the tridiagonal matrix,
// Z = Q Y with Q = P_0 P_1 ... P_{n-2} the Householder reflectors of the reduction.
//
// Reflectors are applied in blocks of NB from the last block to the first in compact WY
// form (Schreiber & Van Loan 1989): P_{k0} ... P_{k0+nb-1} = I - V T V^H with T upper
// triangular, T(c, c) = tau_c, T(0:c, c) = -tau_c T(0:c, 0:c) (V(:, 0:c)^H v_c).
// Each CTA owns a slab of BT_CW columns of Z and, per block, forms X = V^H Z, X <- T X,
// Z <- Z - V X by streaming row tiles through shared memory.
#include "mmf_internal.h"

#define BT_THREADS 512
#define BT_CW 32      // columns of Z per CTA
#define BT_RT 64      // rows per streamed tile
#define LF_RT 16      // rows per tile in the T-factor kernel

// v_c[r] for reflector k = k0 + c: 0 for r <= k, 1 for r = k+1, A(r, k) below
template <class R, class C>
__device__ __forceinline__ C refl(const C* __restrict__ A, int ld, int k, int r) {
    if (r <= k) return czero<C>();
    if (r == k + 1) return mk(R(1), R(0));
    return A[r + (int64_t)k * ld];
}

// T factor of block bi for every system: one CTA per (block, system)
template <class R>
__global__ void __launch_bounds__(BT_THREADS) k_larft(const MmfDesc* __restrict__ descs,
                                                      const int* __restrict__ idx,
                                                      const typename Cx<R>::T* __restrict__ H,
                                                      const typename Cx<R>::T* __restrict__ taup,
                                                      typename Cx<R>::T* __restrict__ Tf) {
    typedef typename Cx<R>::T C;
    __shared__ C G[MMF_NB][MMF_NB + 1];
    __shared__ C Ts[MMF_NB][MMF_NB + 1];
    __shared__ C tile[LF_RT][MMF_NB + 1];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, ld = d.ld;
    const int nref = n - 1;
    const int k0 = blockIdx.x * MMF_NB;
    if (k0 >= nref) return;
    const int nbk = min(MMF_NB, nref - k0);
    const C* A = H + d.mat_off;
    const C* tau = taup + d.vec_off;
    const int tid = threadIdx.x;
    // Gram matrix G = V^H V (nbk x nbk) over rows k0+1 .. n-1
    const int a = tid & 31, b = tid >> 5;  // (a, b) and (a, b + 16)
    C g0 = czero<C>(), g1 = czero<C>();
    for (int r0 = k0 + 1; r0 < n; r0 += LF_RT) {
        for (int e = tid; e < LF_RT * MMF_NB; e += BT_THREADS) {
            int c = e / LF_RT, rr = e - c * LF_RT;
            int r = r0 + rr;
            tile[rr][c] = (r < n && c < nbk) ? refl<R>(A, ld, k0 + c, r) : czero<C>();
        }
        __syncthreads();
        for (int rr = 0; rr < LF_RT; ++rr) {
            C va = tile[rr][a];
            g0 = g0 + cmulc(va, tile[rr][b]);
            g1 = g1 + cmulc(va, tile[rr][b + 16]);
        }
        __syncthreads();
    }
    G[a][b] = g0;
    G[a][b + 16] = g1;
    for (int e = tid; e < MMF_NB * MMF_NB; e += BT_THREADS) Ts[e / MMF_NB][e % MMF_NB] = czero<C>();
    __syncthreads();
    // T(0:c, c) = -tau_c T(0:c, 0:c) G(0:c, c)
    for (int c = 0; c < nbk; ++c) {
        const C tc = tau[k0 + c];
        if (tid < c) {
            C s = czero<C>();
            for (int q = tid; q < c; ++q) s = s + Ts[tid][q] * G[q][c];
            Ts[tid][c] = mk(-(tc.x * s.x - tc.y * s.y), -(tc.x * s.y + tc.y * s.x));
        }
        if (tid == 0) Ts[c][c] = tc;
        __syncthreads();
    }
    C* To = Tf + d.pan_off + (int64_t)blockIdx.x * MMF_NB * MMF_NB;
    for (int e = tid; e < MMF_NB * MMF_NB; e += BT_THREADS) To[e] = Ts[e / MMF_NB][e % MMF_NB];
}

template <class R>
__global__ void __launch_bounds__(BT_THREADS) k_backtransform(
    const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
    const typename Cx<R>::T* __restrict__ H, const typename Cx<R>::T* __restrict__ Tf,
    const double* __restrict__ Yg, typename Cx<R>::T* __restrict__ Zg) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char bt_smem[];
    C(*Vt)[MMF_NB + 1] = reinterpret_cast<C(*)[MMF_NB + 1]>(bt_smem);
    C(*Zt)[BT_CW + 1] = reinterpret_cast<C(*)[BT_CW + 1]>(Vt + BT_RT);
    C(*X)[BT_CW + 1] = reinterpret_cast<C(*)[BT_CW + 1]>(Zt + BT_RT);
    C(*Ts)[MMF_NB + 1] = reinterpret_cast<C(*)[MMF_NB + 1]>(X + MMF_NB);
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, ld = d.ld;
    const int c0 = blockIdx.x * BT_CW;
    if (c0 >= n) return;
    const int ncol = min(BT_CW, n - c0);
    const C* A = H + d.mat_off;
    C* Z = Zg + d.mat_off;
    const double* Y = Yg + d.sq_off;
    const int tid = threadIdx.x;
    // Z(:, slab) = Y(:, slab)
    for (int e = tid; e < n * BT_CW; e += BT_THREADS) {
        int r = e / BT_CW, c = e - r * BT_CW;
        if (c < ncol) Z[r + (int64_t)(c0 + c) * ld] = mk(R(Y[(int64_t)r * n + c0 + c]), R(0));
    }
    __syncthreads();
    const int nref = n - 1;
    const int nblk = (nref + MMF_NB - 1) / MMF_NB;
    const int xp = tid & 31, xc = tid >> 5;  // X(xp, xc) and X(xp, xc + 16)
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int k0 = bi * MMF_NB;
        const int nbk = min(MMF_NB, nref - k0);
        const C* Tb = Tf + d.pan_off + (int64_t)bi * MMF_NB * MMF_NB;
        for (int e = tid; e < MMF_NB * MMF_NB; e += BT_THREADS) Ts[e / MMF_NB][e % MMF_NB] = Tb[e];
        // X = V^H Z over rows k0+1 .. n-1
        C x0 = czero<C>(), x1 = czero<C>();
        for (int r0 = k0 + 1; r0 < n; r0 += BT_RT) {
            for (int e = tid; e < BT_RT * MMF_NB; e += BT_THREADS) {
                int c = e / BT_RT, rr = e - c * BT_RT;
                int r = r0 + rr;
                Vt[rr][c] = (r < n && c < nbk) ? refl<R>(A, ld, k0 + c, r) : czero<C>();
            }
            for (int e = tid; e < BT_RT * BT_CW; e += BT_THREADS) {
                int c = e / BT_RT, rr = e - c * BT_RT;
                int r = r0 + rr;
                Zt[rr][c] = (r < n && c < ncol) ? Z[r + (int64_t)(c0 + c) * ld] : czero<C>();
            }
            __syncthreads();
#pragma unroll 4
            for (int rr = 0; rr < BT_RT; ++rr) {
                C v = Vt[rr][xp];
                x0 = x0 + cmulc(v, Zt[rr][xc]);
                x1 = x1 + cmulc(v, Zt[rr][xc + 16]);
            }
            __syncthreads();
        }
        X[xp][xc] = x0;
        X[xp][xc + 16] = x1;
        __syncthreads();
        // X <- T X
        C y0 = czero<C>(), y1 = czero<C>();
        for (int q = xp; q < MMF_NB; ++q) {
            C t = Ts[xp][q];
            y0 = y0 + t * X[q][xc];
            y1 = y1 + t * X[q][xc + 16];
        }
        __syncthreads();
        X[xp][xc] = y0;
        X[xp][xc + 16] = y1;
        __syncthreads();
        // Z <- Z - V X
        for (int r0 = k0 + 1; r0 < n; r0 += BT_RT) {
            for (int e = tid; e < BT_RT * MMF_NB; e += BT_THREADS) {
                int c = e / BT_RT, rr = e - c * BT_RT;
                int r = r0 + rr;
                Vt[rr][c] = (r < n && c < nbk) ? refl<R>(A, ld, k0 + c, r) : czero<C>();
            }
            __syncthreads();
            for (int e = tid; e < BT_RT * BT_CW; e += BT_THREADS) {
                int c = e / BT_RT, rr = e - c * BT_RT;
                int r = r0 + rr;
                if (r < n && c < ncol) {
                    C acc = czero<C>();
#pragma unroll 8
                    for (int p = 0; p < MMF_NB; ++p) acc = acc + Vt[rr][p] * X[p][c];
                    C* pz = Z + r + (int64_t)(c0 + c) * ld;
                    *pz = *pz - acc;
                }
            }
            __syncthreads();
        }
    }
}

// FP32 variant arranged for the FP32 pipes rather than shared-memory bandwidth: lane = column
// of the slab, so the reflector entries are shared-memory broadcasts and each thread keeps
// several outputs in registers.  Z tiles of BF_RT rows pass through shared memory so that global
// accesses stay coalesced.
//   X = V^H Z:  thread (group g, warp w < 8, lane c): X(4w .. 4w+3, c) over the tile rows of
//               parity g; the two groups' partial sums are added at the end.
//   X <- T X:   thread (w, c): X(w, c), X(w + 16, c).
//   Z -= V X:   thread (w, c): rows 8w .. 8w+7 of column c.
#define BF_RT 128

__global__ void __launch_bounds__(BT_THREADS) k_backtransform_f32(
    const MmfDesc* __restrict__ descs, const int* __restrict__ idx, const float2* __restrict__ H,
    const float2* __restrict__ Tf, const double* __restrict__ Yg, float2* __restrict__ Zg) {
    extern __shared__ __align__(16) unsigned char bf_smem[];
    float2(*Vt)[MMF_NB + 1] = reinterpret_cast<float2(*)[MMF_NB + 1]>(bf_smem);      // BF_RT rows
    float2(*Zt)[BT_CW + 1] = reinterpret_cast<float2(*)[BT_CW + 1]>(Vt + BF_RT);     // BF_RT rows
    float2(*X)[BT_CW] = reinterpret_cast<float2(*)[BT_CW]>(Zt + BF_RT);              // MMF_NB rows
    float2(*Xp)[BT_CW] = X + MMF_NB;                                                 // MMF_NB rows
    float2(*Ts)[MMF_NB + 1] = reinterpret_cast<float2(*)[MMF_NB + 1]>(Xp + MMF_NB);  // MMF_NB rows
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, ld = d.ld;
    const int c0 = blockIdx.x * BT_CW;
    if (c0 >= n) return;
    const int ncol = min(BT_CW, n - c0);
    const float2* A = H + d.mat_off;
    float2* Z = Zg + d.mat_off;
    const double* Y = Yg + d.sq_off;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // Z(:, slab) = Y(:, slab)
    for (int e = tid; e < n * BT_CW; e += BT_THREADS) {
        const int r = e / BT_CW, c = e - r * BT_CW;
        if (c < ncol) Z[r + (int64_t)(c0 + c) * ld] = make_float2((float)Y[(int64_t)r * n + c0 + c], 0.f);
    }
    __syncthreads();
    const int nref = n - 1;
    const int nblk = (nref + MMF_NB - 1) / MMF_NB;
    const int g = warp >> 3, w8 = warp & 7;
    auto load_tiles = [&](int k0, int nbk, int r0) {
        for (int e = tid; e < BF_RT * MMF_NB; e += BT_THREADS) {
            const int c = e / BF_RT, rr = e - c * BF_RT, r = r0 + rr;
            Vt[rr][c] = (r < n && c < nbk) ? refl<float>(A, ld, k0 + c, r) : make_float2(0.f, 0.f);
        }
        for (int e = tid; e < BF_RT * BT_CW; e += BT_THREADS) {
            const int c = e / BF_RT, rr = e - c * BF_RT, r = r0 + rr;
            Zt[rr][c] = (r < n && c < ncol) ? Z[r + (int64_t)(c0 + c) * ld] : make_float2(0.f, 0.f);
        }
    };
    for (int bi = nblk - 1; bi >= 0; --bi) {
        const int k0 = bi * MMF_NB;
        const int nbk = min(MMF_NB, nref - k0);
        const float2* Tb = Tf + d.pan_off + (int64_t)bi * MMF_NB * MMF_NB;
        for (int e = tid; e < MMF_NB * MMF_NB; e += BT_THREADS) Ts[e / MMF_NB][e % MMF_NB] = Tb[e];
        // X = V^H Z over rows k0+1 .. n-1
        float2 x[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = make_float2(0.f, 0.f);
        for (int r0 = k0 + 1; r0 < n; r0 += BF_RT) {
            load_tiles(k0, nbk, r0);
            __syncthreads();
#pragma unroll 4
            for (int rr = g; rr < BF_RT; rr += 2) {
                const float2 z = Zt[rr][lane];
#pragma unroll
                for (int q = 0; q < 4; ++q) x[q] = x[q] + cmulc(Vt[rr][4 * w8 + q], z);
            }
            __syncthreads();
        }
        if (g == 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) Xp[4 * w8 + q][lane] = x[q];
        }
        __syncthreads();
        if (g == 0) {
#pragma unroll
            for (int q = 0; q < 4; ++q) X[4 * w8 + q][lane] = x[q] + Xp[4 * w8 + q][lane];
        }
        __syncthreads();
        // X <- T X (T upper triangular)
        float2 y0 = make_float2(0.f, 0.f), y1 = make_float2(0.f, 0.f);
        for (int q = warp; q < MMF_NB; ++q) y0 = y0 + Ts[warp][q] * X[q][lane];
        for (int q = warp + 16; q < MMF_NB; ++q) y1 = y1 + Ts[warp + 16][q] * X[q][lane];
        __syncthreads();
        X[warp][lane] = y0;
        X[warp + 16][lane] = y1;
        __syncthreads();
        // Z <- Z - V X
        for (int r0 = k0 + 1; r0 < n; r0 += BF_RT) {
            load_tiles(k0, nbk, r0);
            __syncthreads();
            float2 acc[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[q] = make_float2(0.f, 0.f);
#pragma unroll 4
            for (int p = 0; p < MMF_NB; ++p) {
                const float2 xv = X[p][lane];
#pragma unroll
                for (int q = 0; q < 8; ++q) acc[q] = acc[q] + Vt[8 * warp + q][p] * xv;
            }
#pragma unroll
            for (int q = 0; q < 8; ++q) Zt[8 * warp + q][lane] = Zt[8 * warp + q][lane] - acc[q];
            __syncthreads();
            for (int e = tid; e < BF_RT * BT_CW; e += BT_THREADS) {
                const int c = e / BF_RT, rr = e - c * BF_RT, r = r0 + rr;
                if (r < n && c < ncol) Z[r + (int64_t)(c0 + c) * ld] = Zt[rr][c];
            }
            __syncthreads();
        }
    }
}

template <class R>
__global__ void k_widen(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                        const typename Cx<R>::T* __restrict__ Zp, double2* __restrict__ Z) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int64_t tot = (int64_t)d.n * d.ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot;
         e += (int64_t)gridDim.x * blockDim.x)
        Z[d.mat_off + e] = to_c128(Zp[d.mat_off + e]);
}

cudaError_t mmf_launch_backtransform(const MmfLaunch& L, const void* H, const void* tau, void* Tf,
                                     const double* Y, void* Z, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    const int nblk = (L.nmax - 1 + MMF_NB - 1) / MMF_NB;
    dim3 gt(nblk > 0 ? nblk : 1, L.count);
    dim3 gb((L.nmax + BT_CW - 1) / BT_CW, L.count);
    const size_t cs = fp32 ? 8 : 16;
    const size_t sm = cs * (size_t)(BT_RT * (MMF_NB + 1) + BT_RT * (BT_CW + 1) +
                                    MMF_NB * (BT_CW + 1) + MMF_NB * (MMF_NB + 1));
    cudaError_t err;
    if (fp32) {
        const size_t smf = sizeof(float2) * (size_t)(BF_RT * (MMF_NB + 1) + BF_RT * (BT_CW + 1) +
                                                     2 * MMF_NB * BT_CW + MMF_NB * (MMF_NB + 1));
        err = cudaFuncSetAttribute(k_backtransform_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smf);
        if (err != cudaSuccess) return err;
        k_larft<float><<<gt, BT_THREADS, 0, L.stream>>>(L.desc, L.idx, (const float2*)H,
                                                        (const float2*)tau, (float2*)Tf);
        k_backtransform_f32<<<gb, BT_THREADS, smf, L.stream>>>(L.desc, L.idx, (const float2*)H,
                                                              (const float2*)Tf, Y, (float2*)Z);
    } else {
        err = cudaFuncSetAttribute(k_backtransform<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_larft<double><<<gt, BT_THREADS, 0, L.stream>>>(L.desc, L.idx, (const double2*)H,
                                                         (const double2*)tau, (double2*)Tf);
        k_backtransform<double><<<gb, BT_THREADS, sm, L.stream>>>(L.desc, L.idx, (const double2*)H,
                                                                  (const double2*)Tf, Y, (double2*)Z);
    }
    return cudaGetLastError();
}

cudaError_t mmf_launch_widen(const MmfLaunch& L, const void* Zp, double2* Z, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    if (!fp32) return cudaSuccess;
    k_widen<float><<<dim3(256, L.count), 256, 0, L.stream>>>(L.desc, L.idx, (const float2*)Zp, Z);
    return cudaGetLastError();
}
