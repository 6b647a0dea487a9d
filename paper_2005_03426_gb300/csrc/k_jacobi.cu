// k_jacobi.cu -- S2': batched full eigendecomposition of small H_F in shared memory.
//
// One CTA per system: the whole n x n Hermitian matrix A and the accumulated rotations V
// live in shared memory.  Two-sided complex Jacobi with the parallel round-robin
// (Brent & Luk 1985) ordering: each round annihilates n/2 disjoint pivots (p, q) at once,
// A <- J^H A J, V <- V J with J = diag(1, e^{-i phi}) G per pivot, where a_pq = |a_pq| e^{i phi}
// and G = [[c, s], [-s, c]] the symmetric Schur rotation of [[a_pp, |a_pq|], [|a_pq|, a_qq]]
// (Rutishauser's formulas).  A sweep is n-1 rounds; sweeps stop when no pivot exceeds
// eps * ||A||_F.  Output: eigenvalues ascending (ties by index) and the matching columns
// of V.  The paper delegates this step to LAPACK (Sec. 3.2); any exact diagonalisation
// yields the same eigenpairs.
#include "mmf_internal.h"

template <class R> struct JEps;
template <> struct JEps<double> { static constexpr double v = 2.220446049250313e-16; };
template <> struct JEps<float> { static constexpr float v = 1.1920929e-07f; };

template <class R>
__global__ void __launch_bounds__(512) k_jacobi(const MmfDesc* __restrict__ descs,
                                                const int* __restrict__ idx,
                                                const typename Cx<R>::T* __restrict__ H,
                                                double* __restrict__ Eout,
                                                double2* __restrict__ Zout,
                                                int* __restrict__ status, int max_sweeps) {
    typedef typename Cx<R>::T C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int sid = idx[blockIdx.x];
    const MmfDesc d = descs[sid];
    const int n = d.n;
    const int m = (n + 1) & ~1;  // padded to even for the tournament
    C* A = reinterpret_cast<C*>(smem_raw);           // n x n, column-major, lda = n
    C* V = A + (size_t)n * n;                         // n x n
    R* rc = reinterpret_cast<R*>(V + (size_t)n * n);  // per pivot: c, s, cos phi, sin phi
    int* pq = reinterpret_cast<int*>(rc + 4 * (m / 2));
    int* flag = pq + m;
    R* red = reinterpret_cast<R*>(flag + 4);
    const int tid = threadIdx.x, T = blockDim.x;

    const C* Hg = H + d.mat_off;
    for (int e = tid; e < n * n; e += T) {
        int c = e / n, r = e - c * n;
        A[e] = Hg[(int64_t)c * d.ld + r];
        V[e] = (r == c) ? mk(R(1), R(0)) : mk(R(0), R(0));
    }
    // ||A||_F
    R part = 0;
    for (int e = tid; e < n * n; e += T) part += abs2(A[e]);
    part = warp_sum(part);
    if ((tid & 31) == 0) red[tid >> 5] = part;
    __syncthreads();
    if (tid == 0) {
        R s = 0;
        for (int w = 0; w < T / 32; ++w) s += red[w];
        red[32] = sqrt(s) * JEps<R>::v;
    }
    __syncthreads();
    const R thr = red[32];

    int sweep = 0, converged = 0;
    for (; sweep < max_sweeps; ++sweep) {
        if (tid == 0) flag[0] = 0;
        __syncthreads();
        for (int round = 0; round < m - 1; ++round) {
            // pivots of this round: position 0 fixed, the others rotate
            for (int k = tid; k < m / 2; k += T) {
                int a = (k == 0) ? 0 : ((k - 1 + round) % (m - 1)) + 1;
                int kb = m - 1 - k;
                int b = ((kb - 1 + round) % (m - 1)) + 1;
                int p = a < b ? a : b, q = a < b ? b : a;
                pq[2 * k] = p;
                pq[2 * k + 1] = q;
                R c = 1, s = 0, cf = 1, sf = 0;
                if (q < n) {
                    C apq = A[(size_t)q * n + p];
                    R r = sqrt(abs2(apq));
                    if (r > thr) {
                        R app = A[(size_t)p * n + p].x, aqq = A[(size_t)q * n + q].x;
                        cf = apq.x / r;
                        sf = apq.y / r;
                        R theta = (aqq - app) / (R(2) * r);
                        R t = (theta >= R(0) ? R(1) : R(-1)) / (fabs(theta) + sqrt(R(1) + theta * theta));
                        c = R(1) / sqrt(R(1) + t * t);
                        s = t * c;
                        flag[0] = 1;
                    }
                }
                rc[4 * k] = c; rc[4 * k + 1] = s; rc[4 * k + 2] = cf; rc[4 * k + 3] = sf;
            }
            __syncthreads();
            // columns: A <- A J   (J_pp = c, J_pq = s, J_qp = -s e^{-i phi}, J_qq = c e^{-i phi})
            for (int e = tid; e < (m / 2) * n; e += T) {
                int k = e / n, r = e - k * n;
                int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= n) continue;
                R c = rc[4 * k], s = rc[4 * k + 1];
                if (s == R(0) && c == R(1)) continue;
                C em = mk(rc[4 * k + 2], -rc[4 * k + 3]);  // e^{-i phi}
                C ap = A[(size_t)p * n + r], aq = A[(size_t)q * n + r];
                C aqe = aq * em;
                A[(size_t)p * n + r] = c * ap - s * aqe;
                A[(size_t)q * n + r] = s * ap + c * aqe;
                C vp = V[(size_t)p * n + r], vq = V[(size_t)q * n + r];
                C vqe = vq * em;
                V[(size_t)p * n + r] = c * vp - s * vqe;
                V[(size_t)q * n + r] = s * vp + c * vqe;
            }
            __syncthreads();
            // rows: A <- J^H A   (row p' = c row_p - s e^{i phi} row_q, row q' = s row_p + c e^{i phi} row_q)
            for (int e = tid; e < (m / 2) * n; e += T) {
                int k = e / n, col = e - k * n;
                int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= n) continue;
                R c = rc[4 * k], s = rc[4 * k + 1];
                if (s == R(0) && c == R(1)) continue;
                C ep = mk(rc[4 * k + 2], rc[4 * k + 3]);  // e^{+i phi}
                C ap = A[(size_t)col * n + p], aq = A[(size_t)col * n + q];
                C aqe = ep * aq;
                A[(size_t)col * n + p] = c * ap - s * aqe;
                A[(size_t)col * n + q] = s * ap + c * aqe;
            }
            __syncthreads();
            // the pivots are annihilated in exact arithmetic
            for (int k = tid; k < m / 2; k += T) {
                int p = pq[2 * k], q = pq[2 * k + 1];
                if (q >= n || (rc[4 * k + 1] == R(0) && rc[4 * k] == R(1))) continue;
                A[(size_t)q * n + p] = mk(R(0), R(0));
                A[(size_t)p * n + q] = mk(R(0), R(0));
                A[(size_t)p * n + p].y = R(0);
                A[(size_t)q * n + q].y = R(0);
            }
            __syncthreads();
        }
        int any = flag[0];
        __syncthreads();
        if (!any) { converged = 1; break; }
    }

    // eigenvalues ascending, ties by index: rank by counting
    double* E = Eout + d.vec_off;
    double2* Z = Zout + d.mat_off;
    for (int i = tid; i < n; i += T) {
        R di = A[(size_t)i * n + i].x;
        int rank = 0;
        for (int j = 0; j < n; ++j) {
            R dj = A[(size_t)j * n + j].x;
            rank += (dj < di) || (dj == di && j < i);
        }
        pq[i] = rank;  // reuse (m >= n)
    }
    __syncthreads();
    for (int i = tid; i < n; i += T) E[pq[i]] = (double)A[(size_t)i * n + i].x;
    for (int e = tid; e < n * n; e += T) {
        int c = e / n, r = e - c * n;
        Z[(int64_t)pq[c] * d.ld + r] = to_c128(V[e]);
    }
    if (tid == 0) status[sid] = converged ? MMF_ST_OK : MMF_ST_NOCONV;
}

static size_t jacobi_smem(int n, int fp32) {
    int m = (n + 1) & ~1;
    size_t cs = fp32 ? 8 : 16, rs = fp32 ? 4 : 8;
    return 2 * (size_t)n * n * cs + 4 * (m / 2) * rs + (m + 4) * sizeof(int) + 40 * rs + 16;
}

cudaError_t mmf_launch_jacobi(const MmfLaunch& L, void* H, void* Zw, double* E, void* Z,
                              int* status, int fp32, int max_sweeps) {
    (void)Zw;
    if (L.count <= 0) return cudaSuccess;
    size_t sm = jacobi_smem(L.nmax, fp32);
    if (sm > 227 * 1024) return cudaErrorInvalidValue;
    cudaError_t err;
    if (fp32) {
        err = cudaFuncSetAttribute(k_jacobi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_jacobi<float><<<L.count, 512, sm, L.stream>>>(L.desc, L.idx, (const float2*)H, E,
                                                        (double2*)Z, status, max_sweeps);
    } else {
        err = cudaFuncSetAttribute(k_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (err != cudaSuccess) return err;
        k_jacobi<double><<<L.count, 512, sm, L.stream>>>(L.desc, L.idx, (const double2*)H, E,
                                                         (double2*)Z, status, max_sweeps);
    }
    return cudaGetLastError();
}
