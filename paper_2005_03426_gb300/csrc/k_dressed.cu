// k_dressed.cu -- evolution in the dressed basis of a subset of the drive modes (Sec. 3.3, Eq. 4).
//
// A batch of systems restricted to their dressing modes has been diagonalised; for each system s
// its micromotion operator for one Floquet zone (Eq. 5) is
//     U_F(t)[j][a] = sum_b e^{-i (n_b . omega) t} Z_d[(j, b), r_a],
// with r_a the zone representatives (the D eigenvectors of largest central-block weight, ties to
// the lower index, in ascending order) and Ebar_a = E_d[r_a] their quasienergies.  With U(t2, t1)
// of the full system (every mode driving, Eq. 3-4, times t2_k from the common start t1), the
// evolution in the time-dependent dressed basis is
//     Ud_k = U_F(t2_k)^dagger U(t2_k, t1) U_F(t1).
// All in FP64; the work is D^2 M per micromotion entry and 2 D^3 per time, far below the
// eigensolver's.
#include "mmf_internal.h"

// Zone representatives and their quasienergies, one CTA per system of the dressing batch.
__global__ void __launch_bounds__(512) k_dress_zone(const MmfDesc* __restrict__ descs,
                                                   const double2* __restrict__ Zg,
                                                   const double* __restrict__ Eg,
                                                   const int64_t* __restrict__ roff,
                                                   int64_t* __restrict__ reps, double* __restrict__ Ebar) {
    extern __shared__ __align__(16) double wsm[];
    const int s = blockIdx.x;
    const MmfDesc d = descs[s];
    const int n = d.n, D = d.D;
    const double2* Z = Zg + d.mat_off;
    int* sel = reinterpret_cast<int*>(wsm + n);
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        double a = 0.0;
        for (int i = 0; i < D; ++i) a += abs2(Z[(int64_t)l * d.ld + i + D * d.b0]);
        wsm[l] = a;
    }
    __syncthreads();
    // rank of column l by (weight descending, index ascending); the D best are selected
    for (int l = threadIdx.x; l < n; l += blockDim.x) {
        const double wl = wsm[l];
        int rank = 0;
        for (int m = 0; m < n && rank < D; ++m) rank += (wsm[m] > wl) || (wsm[m] == wl && m < l);
        if (rank < D) sel[rank] = l;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 1; a < D; ++a) {  // ascending eigenvalue index
            int v = sel[a], b = a - 1;
            while (b >= 0 && sel[b] > v) { sel[b + 1] = sel[b]; --b; }
            sel[b + 1] = v;
        }
        for (int a = 0; a < D; ++a) {
            reps[roff[s] + a] = sel[a];
            Ebar[roff[s] + a] = Eg[d.vec_off + sel[a]];
        }
    }
}

// U_F at the nt + 1 times {t1, t2_0, ..., t2_{nt-1}} of system s (grid.y = s):
// UF[ufoff[s] + (tau D + j) D + a]
__global__ void k_dress_uf(const MmfDesc* __restrict__ ddesc, const MmfDesc* __restrict__ fdesc,
                           const double2* __restrict__ Zg, const int64_t* __restrict__ reps,
                           const int64_t* __restrict__ roff, const int64_t* __restrict__ ufoff,
                           const double* __restrict__ tg, double t1, int nt, double2* __restrict__ UF) {
    const int s = blockIdx.y;
    const MmfDesc d = ddesc[s];
    const int D = d.D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (nt + 1) * D * D) return;
    const int tau = e / (D * D), j = (e / D) % D, a = e % D;
    const double t = tau == 0 ? t1 : tg[fdesc[s].t_off + tau - 1];
    const double2* z = Zg + d.mat_off + reps[roff[s] + a] * (int64_t)d.ld;
    double2 acc = make_double2(0.0, 0.0);
    for (int b = 0; b < d.M; ++b) {
        double sn, cs;
        sincos(block_ndotw(d, b) * t, &sn, &cs);
        acc = acc + make_double2(cs, -sn) * z[j + D * b];
    }
    UF[ufoff[s] + e] = acc;
}

// W_k = U(t2_k, t1) U_F(t1): W[u_off + (k D + j) D + c] = sum_i U[k][j][i] UF1[i][c]
__global__ void k_dress_w(const MmfDesc* __restrict__ fdesc, const double2* __restrict__ U,
                          const double2* __restrict__ UF, const int64_t* __restrict__ ufoff, int nt,
                          double2* __restrict__ Wt) {
    const int s = blockIdx.y;
    const MmfDesc d = fdesc[s];
    const int D = d.D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt * D * D) return;
    const int k = e / (D * D), j = (e / D) % D, c = e % D;
    const double2* u = U + d.u_off + (int64_t)(k * D + j) * D;
    const double2* f1 = UF + ufoff[s];
    double2 acc = make_double2(0.0, 0.0);
    for (int i = 0; i < D; ++i) acc = acc + u[i] * f1[i * D + c];
    Wt[d.u_off + e] = acc;
}

// Ud_k = U_F(t2_k)^dagger W_k: Ud[u_off + (k D + a) D + c] = sum_j conj(UF2_k[j][a]) W_k[j][c]
__global__ void k_dress_ud(const MmfDesc* __restrict__ fdesc, const double2* __restrict__ Wt,
                           const double2* __restrict__ UF, const int64_t* __restrict__ ufoff, int nt,
                           double2* __restrict__ Ud) {
    const int s = blockIdx.y;
    const MmfDesc d = fdesc[s];
    const int D = d.D;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt * D * D) return;
    const int k = e / (D * D), a = (e / D) % D, c = e % D;
    const double2* f2 = UF + ufoff[s] + (int64_t)(k + 1) * D * D;
    const double2* w = Wt + d.u_off + (int64_t)k * D * D;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = 0; j < D; ++j) acc = acc + cmulc(f2[j * D + a], w[j * D + c]);
    Ud[d.u_off + e] = acc;
}

cudaError_t mmf_launch_dressed(const MmfDesc* ddesc, const MmfDesc* fdesc, int count, int nmax_d, int Dmax,
                               const double2* Zd, const double* Ed, const double2* U, const double* t, double t1,
                               int nt, const int64_t* roff, const int64_t* ufoff, int64_t* reps, double* Ebar,
                               double2* UF, double2* Wt, double2* Ud, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const size_t sm = sizeof(double) * (size_t)nmax_d + sizeof(int) * (size_t)Dmax + 16;
    if (sm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_dress_zone, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
    }
    k_dress_zone<<<count, 512, sm, st>>>(ddesc, Zd, Ed, roff, reps, Ebar);
    const int tot_uf = (nt + 1) * Dmax * Dmax, tot = nt * Dmax * Dmax;
    k_dress_uf<<<dim3((tot_uf + 127) / 128, count), 128, 0, st>>>(ddesc, fdesc, Zd, reps, roff, ufoff, t, t1, nt, UF);
    if (nt > 0) {
        k_dress_w<<<dim3((tot + 127) / 128, count), 128, 0, st>>>(fdesc, U, UF, ufoff, nt, Wt);
        k_dress_ud<<<dim3((tot + 127) / 128, count), 128, 0, st>>>(fdesc, Wt, UF, ufoff, nt, Ud);
    }
    return cudaGetLastError();
}
