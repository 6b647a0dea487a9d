// k_assemble.cu -- S1: dense Floquet matrix H_F of each system in the batch.
//
// Eq. 6 of arXiv 2005.03426 (second coupling index read as U^{n-m}) in the block layout
// of Appendix A: Fourier block b has vector n_k = (b / S_k) mod (2N_k+1) - N_k, mode 1
// innermost; row (i, b), column (j, b') of H_F holds
//     E_ij - (n.omega) delta_ij                    if b' == b
//     V^{l,h}_ij                                   if n(b') - n(b) == +h e_l
//     conj(V^{l,h}_ji)                             if n(b') - n(b) == -h e_l
//     0                                            otherwise.
// The full matrix (both triangles) is written column-major.  The diagonal shift is
// accumulated over modes in ascending order with one rounding per product and sum, so
// the FP64 result is bit-identical to a plain evaluation of that expression; the FP32
// variant rounds each FP64 entry once to nearest.
#include "mmf_internal.h"

template <class C>
__global__ void __launch_bounds__(256) k_assemble(const MmfDesc* __restrict__ descs,
                                                  const int* __restrict__ idx,
                                                  const double2* __restrict__ coef,
                                                  C* __restrict__ H) {
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, D = d.D;
    C* A = H + d.mat_off;
    const double2* H0 = coef + d.coef_off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // one warp per column, lanes over rows
    for (int c = blockIdx.x * 8 + warp; c < n; c += gridDim.x * 8) {
        const int bc = c / D, j = c - bc * D;
        int nvc[MMF_MAX_MODES];
        block_nvec(d, bc, nvc);
        for (int r = lane; r < n; r += 32) {
            const int br = r / D, i = r - br * D;
            double2 v = make_double2(0.0, 0.0);
            if (br == bc) {
                v = H0[i * D + j];
                if (i == j) v = make_double2(__dsub_rn(v.x, block_ndotw(d, br)), 0.0);
            } else {
                int nvr[MMF_MAX_MODES];
                block_nvec(d, br, nvr);
                int ndiff = 0, l = 0, h = 0;
#pragma unroll
                for (int k = 0; k < MMF_MAX_MODES; ++k)
                    if (k < d.K && nvr[k] != nvc[k]) { ++ndiff; l = k; h = nvc[k] - nvr[k]; }
                if (ndiff == 1) {
                    int ah = h > 0 ? h : -h;
                    if (ah <= d.nharm[l]) {
                        int64_t off = d.coef_off + (int64_t)D * D;  // skip H0
                        for (int k = 0; k < l; ++k) off += (int64_t)d.nharm[k] * D * D;
                        const double2* V = coef + off + (int64_t)(ah - 1) * D * D;
                        if (h > 0) v = V[i * D + j];
                        else { double2 t = V[j * D + i]; v = make_double2(t.x, -t.y); }
                    }
                }
            }
            A[(int64_t)c * d.ld + r] = from_c128<C>(v);
        }
    }
}

cudaError_t mmf_launch_assemble(const MmfLaunch& L, const double2* coef, void* H, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    dim3 grid((L.nmax + 7) / 8, L.count);
    if (grid.x > 4096) grid.x = 4096;
    if (fp32)
        k_assemble<float2><<<grid, 256, 0, L.stream>>>(L.desc, L.idx, coef, (float2*)H);
    else
        k_assemble<double2><<<grid, 256, 0, L.stream>>>(L.desc, L.idx, coef, (double2*)H);
    return cudaGetLastError();
}
