// k_outputs.cu -- S7 time-evolution operator and S8 time-averaged transition probabilities
// from the eigenpairs (E_lambda, Z[:, lambda]) of H_F (FP64).
//
// S7 (Eq. 3-5, Eq. 4 read as U_F(t') Ubar U_F(t)^dagger, summed over all Floquet copies):
//   F[t, b]        = e^{-i (n_b . omega) t}
//   Phi_t[j, l]    = sum_b F[t, b] Z[(j, b), l]
//   U(t, t0)[j, i] = sum_l Phi_t[j, l] e^{-i E_l (t - t0)} conj(Z[(i, b0), l])
// S8 (time and phase average of |U_ji|^2; clusters C of eigenvalues closer than
//   delta = cluster_rel * max|E| are averaged together):
//   Pbar_{i->j} = sum_b sum_C | sum_{l in C} Z[(j, b), l] conj(Z[(i, b0), l]) |^2
#include "mmf_internal.h"

// F is stored pre-split into FP32 pieces (Split) for the double-FP32 contraction below.
__global__ void __launch_bounds__(256) k_phase_table(const MmfDesc* __restrict__ descs,
                                                     const int* __restrict__ idx,
                                                     const double* __restrict__ tpool, int nt,
                                                     Split* __restrict__ F) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int tot = nt * d.M;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gridDim.x * blockDim.x) {
        int t = e / d.M, b = e - t * d.M;
        double arg = block_ndotw(d, b) * tpool[d.t_off + t];
        double s, c;
        sincos(arg, &s, &c);
        F[d.f_off + e] = split(make_double2(c, -s));
    }
}

#define U_TPW 8  // times per warp per pass (8 warps -> 64 times per pass)
#define PB_DSMALL 64  // Pbar in one shared-memory table per system up to this many levels

// Z split once into FP32 pieces, Z = Z1 + Zlo (Z1 = fl32(Z), Zlo = fl32(Z - Z1)), so that the
// contraction below converts nothing on the FP64 pipe.
__global__ void __launch_bounds__(256) k_split_z(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                 const double2* __restrict__ Zg, float2* __restrict__ Z1g,
                                                 float2* __restrict__ Zlog) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int64_t tot = (int64_t)d.n * d.ld;
    const double2* Z = Zg + d.mat_off;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const Split v = split(Z[e]);
        Z1g[d.mat_off + e] = make_float2(v.r1, v.i1);
        Zlog[d.mat_off + e] = make_float2(v.r2, v.i2);
    }
}

// Phi is accumulated FP64-accurately in double-FP32 (the FP64 units of GB300 are ~60x slower
// than its FP32 units); the short contraction with the phases and Z0 is done in FP64.
__global__ void __launch_bounds__(256) k_time_evolution(const MmfDesc* __restrict__ descs,
                                                        const int* __restrict__ idx,
                                                        const double* __restrict__ Eg,
                                                        const double2* __restrict__ Zg,
                                                        const float2* __restrict__ Z1g,
                                                        const float2* __restrict__ Zlog,
                                                        const double* __restrict__ tpool,
                                                        double t0, int nt,
                                                        const Split* __restrict__ F,
                                                        double2* __restrict__ U) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, D = d.D, M = d.M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lam = blockIdx.x * 32 + lane;
    if (blockIdx.x * 32 >= n) return;
    const bool valid = lam < n;
    const double2* Zc = Zg + d.mat_off + (int64_t)(valid ? lam : 0) * d.ld;
    const float2* Z1c = Z1g + d.mat_off + (int64_t)(valid ? lam : 0) * d.ld;
    const float2* Zlc = Zlog + d.mat_off + (int64_t)(valid ? lam : 0) * d.ld;
    const double El = valid ? Eg[d.vec_off + lam] : 0.0;
    const Split* Ft = F + d.f_off;
    const double* tt = tpool + d.t_off;
    double2* Uo = U + d.u_off;

    for (int tbase = 0; tbase < nt; tbase += 8 * U_TPW) {
        double2 ph[U_TPW];
#pragma unroll
        for (int q = 0; q < U_TPW; ++q) {
            int t = tbase + warp + 8 * q;
            double s = 0.0, c = 1.0;
            if (t < nt) sincos(El * (tt[t] - t0), &s, &c);
            ph[q] = make_double2(c, -s);
        }
        for (int j = 0; j < D; ++j) {
            DF ar[U_TPW], ai[U_TPW];
#pragma unroll
            for (int q = 0; q < U_TPW; ++q) ar[q] = ai[q] = DF{0.f, 0.f};
            for (int b = 0; b < M; ++b) {
                Split z = Split{0.f, 0.f, 0.f, 0.f};
                if (valid) {
                    const float2 z1 = Z1c[j + D * b], zl = Zlc[j + D * b];
                    z = Split{z1.x, zl.x, z1.y, zl.y};
                }
#pragma unroll
                for (int q = 0; q < U_TPW; ++q) {
                    int t = tbase + warp + 8 * q;
                    if (t < nt) df_cmac(ar[q], ai[q], Ft[(int64_t)t * M + b], z);
                }
                if ((b & 31) == 31) {
#pragma unroll
                    for (int q = 0; q < U_TPW; ++q) { df_renorm(ar[q]); df_renorm(ai[q]); }
                }
            }
            for (int i = 0; i < D; ++i) {
                double2 z0 = valid ? Zc[i + D * d.b0] : make_double2(0.0, 0.0);
#pragma unroll
                for (int q = 0; q < U_TPW; ++q) {
                    int t = tbase + warp + 8 * q;
                    double2 v = cmulc(z0, df_value(ar[q], ai[q]) * ph[q]);  // conj(z0) * Phi * phase
                    v.x = warp_sum(v.x);
                    v.y = warp_sum(v.y);
                    if (lane == 0 && t < nt) {
                        double2* u = Uo + ((int64_t)t * D + j) * D + i;
                        atomicAdd(&u->x, v.x);
                        atomicAdd(&u->y, v.y);
                    }
                }
            }
        }
    }
}

__global__ void __launch_bounds__(256) k_transition_avg(const MmfDesc* __restrict__ descs,
                                                        const int* __restrict__ idx,
                                                        const double* __restrict__ Eg,
                                                        const double2* __restrict__ Zg,
                                                        double cluster_rel,
                                                        double* __restrict__ P) {
    extern __shared__ __align__(16) double psm[];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, D = d.D;
    if (D > PB_DSMALL) return;  // many levels: k_pbar_weights / k_pbar_product / k_pbar_clusters
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double* Ps = psm;                     // D*D
    double* Ws = psm + D * D + warp * D;  // per warp D
    for (int e = threadIdx.x; e < D * D + 8 * D; e += blockDim.x) psm[e] = 0.0;
    __syncthreads();
    const double* E = Eg + d.vec_off;
    const double2* Z = Zg + d.mat_off;
    const double emax = fmax(fabs(E[0]), fabs(E[n - 1]));
    const double delta = cluster_rel * emax;
    const int lam = blockIdx.x * 8 + warp;
    if (lam < n && (lam == 0 || !(E[lam] - E[lam - 1] < delta))) {
        int c1 = lam + 1;
        while (c1 < n && E[c1] - E[c1 - 1] < delta) ++c1;
        if (c1 == lam + 1) {
            const double2* zc = Z + (int64_t)lam * d.ld;
            for (int r = lane; r < n; r += 32) atomicAdd(&Ws[r % D], abs2(zc[r]));
            __syncwarp();
            for (int e = lane; e < D * D; e += 32) {
                int i = e / D, j = e - i * D;
                atomicAdd(&Ps[e], abs2(zc[i + D * d.b0]) * Ws[j]);
            }
        } else {
            for (int r = lane; r < n; r += 32) {
                int j = r % D;
                for (int i = 0; i < D; ++i) {
                    double2 amp = make_double2(0.0, 0.0);
                    for (int l = lam; l < c1; ++l) {
                        const double2* zc = Z + (int64_t)l * d.ld;
                        amp = amp + cmulc(zc[i + D * d.b0], zc[r]);
                    }
                    atomicAdd(&Ps[i * D + j], abs2(amp));
                }
            }
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < D * D; e += blockDim.x)
        if (Ps[e] != 0.0) atomicAdd(&P[d.p_off + e], Ps[e]);
}

// ------------------------------------------------------------------ Pbar for many levels
// Above PB_DSMALL levels the per-system D x D table of k_transition_avg no longer fits shared
// memory (D = 256 for the driven lattice of Sec. 4.2).  The same sum is then split as
//   Pbar_{i->j} = sum_l a_il w_jl  +  sum_{C, |C| >= 2} ( sum_b |sum_{l in C} Z[(j,b),l] conj(Z[(i,b0),l])|^2
//                                                       - sum_{l in C} a_il w_jl )
//   a_il = |Z[(i,b0),l]|^2,   w_jl = sum_b |Z[(j,b),l]|^2
// (the singleton clusters give the first sum).  The first sum is a D x n x D product of
// non-negative terms, tiled in FP64; the cluster terms are added per cluster.  w is kept in a
// scratch slot of D n doubles per system (the H_F slot, free once the eigenvectors exist).
#define PB_T 64   // output tile (i, j)
#define PB_KC 16  // eigenvectors per staged chunk

__device__ __forceinline__ double* pb_w(void* scratch, int esz, const MmfDesc& d) {
    return reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + (size_t)esz * d.mat_off);
}

// w[l * D + j] = sum_b |Z[(j, b), l]|^2; consecutive threads take consecutive j (coalesced in Z)
__global__ void __launch_bounds__(256) k_pbar_weights(const MmfDesc* __restrict__ descs,
                                                      const int* __restrict__ idx,
                                                      const double2* __restrict__ Zg, void* scratch,
                                                      int esz) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    if (d.D <= PB_DSMALL) return;
    const int D = d.D, M = d.M;
    const double2* Z = Zg + d.mat_off;
    double* w = pb_w(scratch, esz, d);
    const int64_t tot = (int64_t)d.n * D;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
        const int l = (int)(e / D), j = (int)(e - (int64_t)l * D);
        const double2* zc = Z + (int64_t)l * d.ld + j;
        double acc = 0.0;
        for (int b = 0; b < M; ++b) acc += abs2(zc[(int64_t)b * D]);
        w[e] = acc;
    }
}

// P[i * D + j] = sum_l a_il w_jl over one 64 x 64 (i, j) tile; 256 threads, 4 x 4 outputs each
__global__ void __launch_bounds__(256) k_pbar_product(const MmfDesc* __restrict__ descs,
                                                      const int* __restrict__ idx,
                                                      const double2* __restrict__ Zg,
                                                      const void* scratch, int esz,
                                                      double* __restrict__ P) {
    __shared__ double As[PB_KC][PB_T];
    __shared__ double Ws[PB_KC][PB_T];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int D = d.D;
    if (D <= PB_DSMALL) return;
    const int ti = blockIdx.y * PB_T, tj = blockIdx.x * PB_T;
    if (ti >= D || tj >= D) return;
    const double2* Z0 = Zg + d.mat_off + (int64_t)D * d.b0;  // central block rows (i, b0)
    const double* w = pb_w(const_cast<void*>(scratch), esz, d);
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.0;
    for (int l0 = 0; l0 < d.n; l0 += PB_KC) {
        for (int e = threadIdx.x; e < PB_KC * PB_T; e += 256) {
            const int k = e / PB_T, r = e - k * PB_T, l = l0 + k;
            const bool ok = l < d.n;
            As[k][r] = (ok && ti + r < D) ? abs2(Z0[(int64_t)l * d.ld + ti + r]) : 0.0;
            Ws[k][r] = (ok && tj + r < D) ? w[(int64_t)l * D + tj + r] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < PB_KC; ++k) {
            double av[4], wv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[k][ty + 16 * a];
#pragma unroll
            for (int c = 0; c < 4; ++c) wv[c] = Ws[k][tx + 16 * c];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][c] = fma(av[a], wv[c], acc[a][c]);
        }
        __syncthreads();
    }
    double* Po = P + d.p_off;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int i = ti + ty + 16 * a;
        if (i >= D) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = tj + tx + 16 * c;
            if (j < D) Po[(int64_t)i * D + j] = acc[a][c];
        }
    }
}

// Cluster terms: one block per leading eigenvalue of a cluster of two or more (gaps < delta).
// With u_il = conj(Z[(i,b0),l]) and S_j(l,l') = sum_b Z[(j,b),l] conj(Z[(j,b),l']), the
// cluster's sum_b |sum_l u_il Z[(j,b),l]|^2 exceeds its diagonal part sum_l a_il w_jl by
//   sum_{l < l'} 2 Re( u_il conj(u_il') S_j(l,l') ),
// which is added pair by pair: S_j in shared memory (D entries), then the D x D pairs of
// levels.  Added after k_pbar_product on the same stream.
__global__ void __launch_bounds__(256) k_pbar_clusters(const MmfDesc* __restrict__ descs,
                                                       const int* __restrict__ idx,
                                                       const double* __restrict__ Eg,
                                                       const double2* __restrict__ Zg, double cluster_rel,
                                                       double* __restrict__ P) {
    extern __shared__ __align__(16) double2 Sj[];  // D entries
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, D = d.D, M = d.M;
    if (D <= PB_DSMALL) return;
    const double* E = Eg + d.vec_off;
    const double delta = cluster_rel * fmax(fabs(E[0]), fabs(E[n - 1]));
    const double2* Z = Zg + d.mat_off;
    const double2* Z0 = Z + (int64_t)D * d.b0;  // central block rows (i, b0)
    for (int lam = blockIdx.x; lam < n; lam += gridDim.x) {
        if (lam > 0 && E[lam] - E[lam - 1] < delta) continue;  // not a cluster's first eigenvalue
        int c1 = lam + 1;
        while (c1 < n && E[c1] - E[c1 - 1] < delta) ++c1;
        for (int l = lam; l < c1; ++l) {
            for (int l2 = l + 1; l2 < c1; ++l2) {
                const double2* za = Z + (int64_t)l * d.ld;
                const double2* zb = Z + (int64_t)l2 * d.ld;
                for (int j = threadIdx.x; j < D; j += blockDim.x) {
                    double2 acc = make_double2(0.0, 0.0);
                    for (int b = 0; b < M; ++b) acc = acc + cmulc(zb[j + D * b], za[j + D * b]);
                    Sj[j] = acc;  // sum_b Z[(j,b),l] conj(Z[(j,b),l2])
                }
                __syncthreads();
                for (int e = threadIdx.x; e < D * D; e += blockDim.x) {
                    const int i = e / D, j = e - i * D;
                    // conj(Z[(i,b0),l]) Z[(i,b0),l2] S_j(l,l2)
                    const double2 uu = cmulc(Z0[(int64_t)l * d.ld + i], Z0[(int64_t)l2 * d.ld + i]);
                    const double2 sj = Sj[j];
                    atomicAdd(&P[d.p_off + e], 2.0 * (uu.x * sj.x - uu.y * sj.y));
                }
                __syncthreads();
            }
        }
    }
}

// Staged launcher with explicit maxima (the batch knows them).
// skip_u: the phase table and the FP32 pieces of Z are prepared, but U is left to the
// tensor-core path (mmf_launch_phi)
cudaError_t mmf_launch_outputs(const MmfLaunch& L, int Mmax, int Dmax, const double* E,
                                  const double2* Z, float2* Z1, float2* Zlo, const double* t, double t0, int nt,
                                  double2* F2, double2* U, double* P, double cluster_rel, int skip_u,
                                  void* scratch, int scratch_esz) {
    static_assert(sizeof(Split) == sizeof(double2), "phase table slots hold one Split each");
    Split* F = reinterpret_cast<Split*>(F2);
    if (L.count <= 0) return cudaSuccess;
    if (nt > 0) {
        int gx = (nt * Mmax + 255) / 256;
        if (gx > 1024) gx = 1024;
        k_phase_table<<<dim3(gx, L.count), 256, 0, L.stream>>>(L.desc, L.idx, t, nt, F);
        k_split_z<<<dim3(128, L.count), 256, 0, L.stream>>>(L.desc, L.idx, Z, Z1, Zlo);
        if (!skip_u)
            k_time_evolution<<<dim3((L.nmax + 31) / 32, L.count), 256, 0, L.stream>>>(
                L.desc, L.idx, E, Z, Z1, Zlo, t, t0, nt, F, U);
    }
    const int Ds = Dmax < PB_DSMALL ? Dmax : PB_DSMALL;
    size_t sm = sizeof(double) * (size_t)(Ds * Ds + 8 * Ds);
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_transition_avg,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_transition_avg<<<dim3((L.nmax + 7) / 8, L.count), 256, sm, L.stream>>>(L.desc, L.idx, E, Z,
                                                                            cluster_rel, P);
    if (Dmax > PB_DSMALL) {
        // scratch holds D n doubles per system at byte offset scratch_esz * mat_off
        if (!scratch || scratch_esz < (int)sizeof(double)) return cudaErrorInvalidValue;
        const int64_t wt = (int64_t)L.nmax * Dmax;
        int gx = (int)((wt + 255) / 256);
        if (gx > 2048) gx = 2048;
        k_pbar_weights<<<dim3(gx, L.count), 256, 0, L.stream>>>(L.desc, L.idx, Z, scratch, scratch_esz);
        const int nt_ = (Dmax + PB_T - 1) / PB_T;
        k_pbar_product<<<dim3(nt_, nt_, L.count), 256, 0, L.stream>>>(L.desc, L.idx, Z, scratch, scratch_esz, P);
        int gc = L.nmax < 1024 ? L.nmax : 1024;
        const size_t smc = sizeof(double2) * (size_t)Dmax;
        if (smc > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k_pbar_clusters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
            if (e != cudaSuccess) return e;
        }
        k_pbar_clusters<<<dim3(gc, L.count), 256, smc, L.stream>>>(L.desc, L.idx, E, Z, cluster_rel, P);
    }
    return cudaGetLastError();
}

// ------------------------------------------------------------------ micromotion (Eq. 5)
// Zone representatives: the D eigenvectors with the largest weight on the central Fourier
// block, w_l = sum_i |Z[(i, b0), l]|^2 (ties to the lower index), returned in ascending order.
__global__ void __launch_bounds__(512) k_zone_select(const MmfDesc* __restrict__ descs,
                                                    const int* __restrict__ idx,
                                                    const double2* __restrict__ Zg,
                                                    int64_t* __restrict__ reps) {
    extern __shared__ __align__(16) double wsm[];
    const MmfDesc d = descs[idx[blockIdx.x]];
    const int n = d.n, D = d.D;
    const double2* Z = Zg + d.mat_off;
    int* sel = reinterpret_cast<int*>(wsm + n);
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        double a = 0.0;
        for (int i = 0; i < D; ++i) a += abs2(Z[(int64_t)l * d.ld + i + D * d.b0]);
        wsm[l] = a;
    }
    __syncthreads();
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const double wl = wsm[l];
        int rank = 0;
        for (int m = 0; m < n && rank < D; ++m) rank += (wsm[m] > wl) || (wsm[m] == wl && m < l);
        if (rank < D) sel[rank] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 1; a < D; ++a) {
            int v = sel[a], b = a - 1;
            while (b >= 0 && sel[b] > v) { sel[b + 1] = sel[b]; --b; }
            sel[b + 1] = v;
        }
        for (int a = 0; a < D; ++a) reps[a] = sel[a];
    }
}

// UF[k][j][a] = sum_b e^{-i (n_b . omega) t_k} Z[(j, b), reps[a]]
__global__ void k_micromotion(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                              const double2* __restrict__ Zg, const int64_t* __restrict__ reps,
                              const double* __restrict__ t, int nt, double2* __restrict__ UF) {
    const MmfDesc d = descs[idx[0]];
    const int D = d.D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt * D * D) return;
    const int k = e / (D * D), j = (e / D) % D, a = e % D;
    const double2* z = Zg + d.mat_off + reps[a] * d.ld;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < d.M; ++b) {
        double s, c;
        sincos(block_ndotw(d, b) * t[k], &s, &c);
        acc = acc + make_double2(c, -s) * z[j + D * b];
    }
    UF[e] = acc;
}

cudaError_t mmf_launch_micromotion(const MmfLaunch& L, int D, const double2* Z, const double* t,
                                   int nt, int64_t* reps, double2* UF) {
    size_t sm = sizeof(double) * (size_t)L.nmax + sizeof(int) * (size_t)D + 16;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_zone_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_zone_select<<<1, 512, sm, L.stream>>>(L.desc, L.idx, Z, reps);
    const int tot = nt * D * D;
    k_micromotion<<<(tot + 127) / 128, 128, 0, L.stream>>>(L.desc, L.idx, Z, reps, t, nt, UF);
    return cudaGetLastError();
}
