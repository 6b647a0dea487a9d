// k_sbr.cu -- S2 for a banded H_F: reduction of the band straight to real tridiagonal form by
// Householder bulge chasing, and the back-transform of the chase's reflectors (S5).
//
// H_F is block-banded (Eq. 6, Appendix A): every nonzero lies within b of the diagonal, with
// b = max over the couplings' nonzero entries V^{l,h}[i][i'] of D h S_l + i' - i (and the width
// of H0).  The dense reduction (k_hetrd) would destroy that structure after one panel; the band
// reduction of Schwarz / Bischof, Lang & Sun keeps the work inside a band of width 2b and costs
// O(n^2 b) instead of O(n^3).  This is the "one column per sweep" chase:
//   sweep j (j = 0 .. n-2), step 0: the reflector H(j,0) of rows R0 = [j+1, j+b] annihilates
//     A(j+2.., j) (A(j+1, j) becomes the real beta = e_j) and is applied from both sides to the
//     diagonal block A(R0, R0);
//   step s >= 1: the previous reflector, applied from the right to the block B = A(Rs, Rs-1)
//     below it (Rs = Rs-1 + b), fills B's lower triangle (the bulge); H(j,s) annihilates B's
//     first column below its first row, is applied from the left to B's other columns and from
//     both sides to A(Rs, Rs).  The rest of the bulge is removed by sweep j+1.
// All reflectors satisfy H^H x = beta e_1 with beta real (H = I - tau v v^H, v[0] = 1; the
// convention of k_hetrd), so T = Q^H H_F Q is real and Q = prod_j prod_s H(j, s).
//
// Pipelining: sweep j+1 may run its step s once sweep j has finished step s+1 (their later
// steps touch disjoint entries), so several sweeps are in flight at once.  One CTA per system;
// NG groups of G threads each take every NG-th sweep, publish their progress in shared memory and
// wait (bounded) for their predecessor's.  A step stages its two b x b blocks in the group's
// shared memory; the band itself stays in the dense matrix's lower triangle (global memory,
// L2-resident: about n x 2b entries are ever touched).
//
// Back-transform: Z = Q Y.  Reflectors of one sweep touch disjoint rows, and H(j', s') must
// precede H(j, s) only if j' > j and s' in {s-1, s}, so the order "s ascending, j descending"
// is valid.  In pass s consecutive reflectors overlap in all but one row: one thread per column
// of Z keeps a window of BMAX rows in registers, applies the reflector (a length-BMAX dot
// product and update), and slides the window up one row.  Z is kept row-major so that the
// threads of a warp (consecutive columns) load and store consecutive addresses.
#include <cooperative_groups.h>
#include <cstdlib>

#include "mmf_internal.h"

namespace cg = cooperative_groups;

// ------------------------------------------------------------------ reflector store
// (layout and Z's place: sbr_off / sbr_zbase in mmf_internal.h)
int64_t mmf_sbr_store_elems(int n, int b) { return sbr_nref(n, b) * (b + 1); }

#define SBR_WAIT_LIMIT (1 << 26)
// bytes before the groups' blocks in dynamic shared memory (progress keys, abort flag), rounded to
// 256 so that the blocks' 16-byte complex elements stay aligned
__host__ __device__ constexpr int sbr_hdr(int ng) { return (8 * ng + 16 + 255) / 256 * 256; }

template <class C, int BMAX, int P>
struct SbrGroup {
    C B[BMAX][BMAX + 1];
    C Dm[BMAX][BMAX + 1];
    C v[2][BMAX];   // current and previous reflector
    C y[BMAX], w[BMAX];
    C red[P][BMAX];
    C tau[2];
    double rs[32];
    int stop;  // the group's copy of the abort flag, taken by its first thread after each wait
    int pad[3];
};

// Asynchronous copy of one complex element global -> shared (8 or 16 bytes); ok = false fills
// zeros without reading (the source address given is then any valid one).
template <class C>
__device__ __forceinline__ void cp_elem(C* sdst, const C* gsrc, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(sdst);
    if (sizeof(C) == 16)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(gsrc), "r"(ok ? 16 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(gsrc), "r"(ok ? 8 : 0) : "memory");
}
// Load of one complex element from L2, bypassing L1: the two CTAs of a cluster run on different
// SMs, whose L1 caches are not coherent, so band data written by one must not be read by the other
// from a stale L1 line.
__device__ __forceinline__ float2 ld_cg(const float2* p) {
    float2 r;
    asm volatile("ld.global.cg.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ double2 ld_cg(const double2* p) {
    double2 r;
    asm volatile("ld.global.cg.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ void cp_wait_all() {
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int G>
__device__ __forceinline__ void gbar(int g) {
    if (G == 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(G) : "memory");
    }
}

// sum over the G threads of the group (every thread gets the result)
template <int G, class R>
__device__ __forceinline__ R group_sum(R v, double* rs, int tid, int g) {
    v = warp_sum(v);
    if (G == 32) return v;
    if ((tid & 31) == 0) rs[tid >> 5] = (double)v;
    gbar<G>(g);
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < G / 32; ++k) s += rs[k];
    gbar<G>(g);
    return (R)s;
}

template <class R> __device__ __forceinline__ R rsqrt_of(R x);
template <> __device__ __forceinline__ float rsqrt_of<float>(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_of<double>(double x) { return sqrt(x); }

// Householder of x = (alpha, rest) with ||rest||^2 = xn2: H^H x = beta e1, beta real.
// Returns tau and beta; scale = 1 / (alpha - beta) multiplies rest into v.
template <class R, class C>
__device__ __forceinline__ void make_reflector(C alpha, R xn2, C& tau, R& beta, C& scale) {
    if (xn2 == R(0) && alpha.y == R(0)) {
        tau = mk(R(0), R(0));
        beta = alpha.x;
        scale = mk(R(0), R(0));
        return;
    }
    const R nrm = rsqrt_of<R>(alpha.x * alpha.x + alpha.y * alpha.y + xn2);
    beta = alpha.x >= R(0) ? -nrm : nrm;
    tau = mk((beta - alpha.x) / beta, -alpha.y / beta);
    const C den = mk(alpha.x - beta, alpha.y);
    const R dd = den.x * den.x + den.y * den.y;
    scale = mk(den.x / dd, -den.y / dd);
}

// Two-sided update A <- H^H A H of the l x l Hermitian block held (both triangles) in Dm, with
// H = I - tau v v^H: y = A v, w = tau y - |tau|^2 (v^H y) / 2 v, A -= v w^H + w v^H; the lower
// triangle is written to global memory at Hg (column-major, ld) from row/column r.
template <class R, class C, int BMAX, int G, int P>
__device__ __forceinline__ void sbr_two_sided(SbrGroup<C, BMAX, P>& S, const C* v, C tau, int l, C* __restrict__ Hg,
                                              int ld, int r, int tid, int g, double* dout) {
    const int i = tid % BMAX, p = tid / BMAX;
    C acc = mk(R(0), R(0)), acc1 = acc;  // two partial sums: independent FMA chains
#pragma unroll
    for (int q = 0; q < BMAX / P; q += 2) {
        acc = acc + S.Dm[i][p + q * P] * v[p + q * P];
        acc1 = acc1 + S.Dm[i][p + (q + 1) * P] * v[p + (q + 1) * P];
    }
    S.red[p][i] = acc + acc1;
    gbar<G>(g);
    R a_part = R(0);
    if (tid < BMAX) {
        C yy = S.red[0][tid];
#pragma unroll
        for (int q = 1; q < P; ++q) yy = yy + S.red[q][tid];
        S.y[tid] = yy;
        const C vv = v[tid];
        a_part = vv.x * yy.x + vv.y * yy.y;  // Re(conj(v) y)
    }
    const R a = group_sum<G, R>(a_part, S.rs, tid, g);
    const R t2 = R(0.5) * (tau.x * tau.x + tau.y * tau.y) * a;
    if (tid < BMAX) S.w[tid] = tau * S.y[tid] - t2 * v[tid];
    gbar<G>(g);
    // lower triangle, column by column (rows i >= k contiguous in global memory)
    const C vi = v[i], wi = S.w[i];
#pragma unroll
    for (int q = 0; q < BMAX / P; ++q) {
        const int k = p + q * P;
        if (i >= k && i < l) {
            const C vk = v[k], wk = S.w[k];
            C a0 = S.Dm[i][k];
            a0 = a0 - cmulc(wk, vi) - cmulc(vk, wi);  // v_i conj(w_k) + w_i conj(v_k)
            if (i == k) {
                a0.y = R(0);
                if (dout && i == 0) *dout = (double)a0.x;
            }
            Hg[(r + k) * ld + r + i] = a0;
        }
    }
}

// CL = 1: one CTA per system.  CL = 2: a cluster of two CTAs (two SMs) per system, the sweeps
// dealt round-robin over both CTAs' groups; a group reads its predecessor's progress key from the
// partner's shared memory (distributed shared memory), the band is read from L2 only (ld.cg), and
// progress is published after a GPU-scope fence.
template <class R, int BMAX, int G, int NG, int CL>
__global__ void __launch_bounds__(G* NG) k_sbr_chase(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                    typename Cx<R>::T* __restrict__ Hbase,
                                                    typename Cx<R>::T* __restrict__ store_base,
                                                    double* __restrict__ dvec, double* __restrict__ evec,
                                                    int* __restrict__ status) {
    typedef typename Cx<R>::T C;
    constexpr int P = G / BMAX;
    static_assert(P * BMAX == G && P >= 1, "group size is a multiple of BMAX");
    constexpr int NGT = CL * NG;                          // groups per system
    constexpr int LCH = (BMAX / P) < 16 ? (BMAX / P) : 16;  // register-staged loads per batch (CL > 1)
    static_assert((BMAX / P) % LCH == 0, "load batches divide the block");
    extern __shared__ __align__(16) unsigned char sbr_smem[];
    volatile long long* key = reinterpret_cast<volatile long long*>(sbr_smem);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(sbr_smem + 8 * NG);
    SbrGroup<C, BMAX, P>* groups = reinterpret_cast<SbrGroup<C, BMAX, P>*>(sbr_smem + sbr_hdr(NG));
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = CL > 1 ? (int)cluster.block_rank() : 0;
    volatile int* abort_peer = abort_flag;
    if (CL > 1) abort_peer = cluster.map_shared_rank(const_cast<int*>(abort_flag), rank ^ 1);

    const int sid = idx[blockIdx.x / CL];
    const MmfDesc d = descs[sid];
    const int n = d.n, b = d.band;
    const int ldi = d.ld;  // in-system offsets fit 32 bits (n ld < 2^31, checked by the host)
    C* Hg = Hbase + d.mat_off;
    // the store lives in the system's FP64 complex matrix slot
    C* V = reinterpret_cast<C*>(store_base + (sizeof(R) == 4 ? 2 : 1) * d.mat_off);
    C* T = V + sbr_nref(n, b) * b;
    double* dd = dvec + d.vec_off;
    double* ee = evec + d.vec_off;
    const int g = threadIdx.x / G, tid = threadIdx.x % G;
    const int gg = rank * NG + g;  // the group's number within the system
    SbrGroup<C, BMAX, P>& S = groups[g];
    const long long KK = sbr_passes(n, b) + 3;
    // the predecessor sweep's group and its progress key (possibly in the partner CTA)
    const int ggp = (gg + NGT - 1) % NGT;
    volatile long long* pkey = key + (ggp % NG);
    if (CL > 1 && ggp / NG != rank)
        pkey = cluster.map_shared_rank(const_cast<long long*>(key), ggp / NG) + (ggp % NG);

    if (threadIdx.x < NG) key[threadIdx.x] = -1;
    if (threadIdx.x == 0) *abort_flag = 0;
    if (CL > 1) cluster.sync(); else __syncthreads();
    if (threadIdx.x == 0 && rank == 0) dd[0] = (double)Hg[0].x;

    const int i = tid % BMAX, p = tid / BMAX;
    int cur = 0;  // buffer of the current reflector in S.v
    bool stopped = false;
    for (int j = gg; j <= n - 2 && !stopped; j += NGT) {
        const int nsteps = (n - 2 - j) / b + 1;
        for (int s = 0; s < nsteps; ++s) {
            // wait until sweep j-1 has finished step s+1 (or all of its steps)
            if (j > 0) {
                if (tid == 0) {
                    const long long need = (long long)(j - 1) * KK + (s + 2 < KK - 1 ? s + 2 : KK - 1);
                    int it = 0;
                    while (*pkey < need && !*abort_flag && !*abort_peer) {
                        if (++it > SBR_WAIT_LIMIT) {
                            *abort_flag = 1;
                            status[sid] = MMF_ST_NOCONV;
                            break;
                        }
                        __nanosleep(64);
                    }
                    if (CL > 1) __threadfence(); else __threadfence_block();
                    S.stop = *abort_flag || *abort_peer;
                }
                gbar<G>(g);
                if (S.stop) {  // the whole group leaves together
                    stopped = true;
                    break;
                }
            }
            const int r = j + 1 + s * b;
            const int l = min(b, n - r);
            C* vc = S.v[cur];
            const C* vp = S.v[cur ^ 1];
            C tau;
            if (s == 0) {
                // column j below the diagonal and the diagonal block, lower triangle
                // all of the step's loads in flight at once (asynchronous copies, zero-filled
                // outside the l x l block)
                if (CL == 1) {
                    if (tid < BMAX) cp_elem(&vc[tid], Hg + j * ldi + r + (tid < l ? tid : 0), tid < l);
#pragma unroll
                    for (int q = 0; q < BMAX / P; ++q) {
                        const int k = p + q * P;
                        const bool ok = i < l && k < l && i >= k;
                        cp_elem(&S.Dm[i][k], Hg + (ok ? (r + k) * ldi + r + i : 0), ok);
                    }
                    cp_wait_all();
                } else {
                    const C z0 = mk(R(0), R(0));
                    if (tid < BMAX) vc[tid] = tid < l ? ld_cg(Hg + j * ldi + r + tid) : z0;
#pragma unroll
                    for (int q0 = 0; q0 < BMAX / P; q0 += LCH) {
                        C rd[LCH];
#pragma unroll
                        for (int u = 0; u < LCH; ++u) {
                            const int k = p + (q0 + u) * P;
                            rd[u] = (i < l && k < l && i >= k) ? ld_cg(Hg + (r + k) * ldi + r + i) : z0;
                        }
#pragma unroll
                        for (int u = 0; u < LCH; ++u) S.Dm[i][p + (q0 + u) * P] = rd[u];
                    }
                }
                gbar<G>(g);
#pragma unroll
                for (int q = 0; q < BMAX / P; ++q) {
                    const int k = p + q * P;
                    if (i < k) S.Dm[i][k] = conj(S.Dm[k][i]);
                }
                const C alpha = vc[0];
                const R xn2 = group_sum<G, R>((tid >= 1 && tid < l) ? abs2(vc[tid]) : R(0), S.rs, tid, g);
                R beta;
                C scale;
                make_reflector<R, C>(alpha, xn2, tau, beta, scale);
                if (tid < BMAX) {
                    const C x = vc[tid];
                    vc[tid] = tid == 0 ? mk(R(1), R(0)) : ((tid < l) ? x * scale : mk(R(0), R(0)));
                    if (tid < l) Hg[j * ldi + r + tid] = tid == 0 ? mk(beta, R(0)) : mk(R(0), R(0));
                }
                if (tid == 0) {
                    ee[j] = (double)beta;
                    S.tau[cur] = tau;
                }
            } else {
                const int rp = r - b;
                const int lp = min(b, n - rp);
                const C taup = S.tau[cur ^ 1];
                if (CL == 1) {
#pragma unroll
                    for (int q = 0; q < BMAX / P; ++q) {
                        const int k = p + q * P;
                        const bool okb = i < l && k < lp, okd = i < l && k < l && i >= k;
                        cp_elem(&S.B[i][k], Hg + (okb ? (rp + k) * ldi + r + i : 0), okb);
                        cp_elem(&S.Dm[i][k], Hg + (okd ? (r + k) * ldi + r + i : 0), okd);
                    }
                    cp_wait_all();
                } else {
                    const C z0 = mk(R(0), R(0));
#pragma unroll
                    for (int q0 = 0; q0 < BMAX / P; q0 += LCH) {
                        C rb[LCH], rd[LCH];
#pragma unroll
                        for (int u = 0; u < LCH; ++u) {
                            const int k = p + (q0 + u) * P;
                            rb[u] = (i < l && k < lp) ? ld_cg(Hg + (rp + k) * ldi + r + i) : z0;
                            rd[u] = (i < l && k < l && i >= k) ? ld_cg(Hg + (r + k) * ldi + r + i) : z0;
                        }
#pragma unroll
                        for (int u = 0; u < LCH; ++u) {
                            S.B[i][p + (q0 + u) * P] = rb[u];
                            S.Dm[i][p + (q0 + u) * P] = rd[u];
                        }
                    }
                }
                gbar<G>(g);
#pragma unroll
                for (int q = 0; q < BMAX / P; ++q) {
                    const int k = p + q * P;
                    if (i < k) S.Dm[i][k] = conj(S.Dm[k][i]);
                }
                // The previous reflector from the right and the new one from the left, as one rank-2
                // update: with C1 = B H(j,s-1) = B - tau_p y v_p^H (y = B v_p), x = C1(:, 0) gives
                // H(j,s); then H^H C1 = B - tau_p y v_p^H - conj(tau) v r with
                // r_k = (v^H B)_k - tau_p (v^H y) conj(v_p,k).
                C acc = mk(R(0), R(0)), acc1 = acc;
#pragma unroll
                for (int q = 0; q < BMAX / P; q += 2) {
                    acc = acc + S.B[i][p + q * P] * vp[p + q * P];
                    acc1 = acc1 + S.B[i][p + (q + 1) * P] * vp[p + (q + 1) * P];
                }
                S.red[p][i] = acc + acc1;
                gbar<G>(g);
                if (tid < BMAX) {
                    C yy = S.red[0][tid];
#pragma unroll
                    for (int q = 1; q < P; ++q) yy = yy + S.red[q][tid];
                    const C ty = taup * yy;
                    S.y[tid] = ty;                      // tau_p y
                    S.w[tid] = S.B[tid][0] - ty;        // x = C1(:, 0)   (v_p[0] = 1)
                }
                gbar<G>(g);
                const C alpha = S.w[0];
                const R xn2 = group_sum<G, R>((tid >= 1 && tid < l) ? abs2(S.w[tid]) : R(0), S.rs, tid, g);
                R beta;
                C scale;
                make_reflector<R, C>(alpha, xn2, tau, beta, scale);
                if (tid < BMAX) {
                    const C x = S.w[tid];
                    vc[tid] = tid == 0 ? mk(R(1), R(0)) : ((tid < l) ? x * scale : mk(R(0), R(0)));
                }
                if (tid == 0) S.tau[cur] = tau;
                gbar<G>(g);
                // u_k = sum_i conj(v_i) B(i, k) and gamma = v^H (tau_p y)
                {
                    const int kc = tid % BMAX, pc = tid / BMAX;
                    C z = mk(R(0), R(0)), z1 = z;
#pragma unroll
                    for (int q = 0; q < BMAX / P; q += 2) {
                        z = z + cmulc(vc[pc + q * P], S.B[pc + q * P][kc]);
                        z1 = z1 + cmulc(vc[pc + (q + 1) * P], S.B[pc + (q + 1) * P][kc]);
                    }
                    S.red[pc][kc] = z + z1;
                }
                gbar<G>(g);
                const R gre = group_sum<G, R>(tid < BMAX ? vc[tid].x * S.y[tid].x + vc[tid].y * S.y[tid].y : R(0),
                                              S.rs, tid, g);
                const R gim = group_sum<G, R>(tid < BMAX ? vc[tid].x * S.y[tid].y - vc[tid].y * S.y[tid].x : R(0),
                                              S.rs, tid, g);
                if (tid < BMAX) {
                    C u = S.red[0][tid];
#pragma unroll
                    for (int q = 1; q < P; ++q) u = u + S.red[q][tid];
                    // r_k = u_k - gamma conj(v_p,k), gamma = v^H (tau_p y); stored conj(tau) r_k
                    const C rk = u - mk(gre, gim) * conj(vp[tid]);
                    S.w[tid] = conj(tau) * rk;
                }
                gbar<G>(g);
                {
                    const C ty = S.y[i], vi = vc[i];
#pragma unroll
                    for (int q = 0; q < BMAX / P; ++q) {
                        const int k = p + q * P;
                        C bk = S.B[i][k] - ty * conj(vp[k]) - vi * S.w[k];
                        if (k == 0) bk = i == 0 ? mk(beta, R(0)) : mk(R(0), R(0));
                        if (i < l && k < lp) Hg[(rp + k) * ldi + r + i] = bk;
                    }
                }
            }
            // store the reflector for the back-transform, marked evict-first: the store is written
            // once and read only after the chase, and L2 should keep the band's lines instead
            if (tid < b) __stcs(&V[(sbr_off(n, b, s) + j) * b + tid], vc[tid]);
            if (tid == 0) __stcs(&T[sbr_off(n, b, s) + j], tau);
            gbar<G>(g);
            // (d) diagonal block A(R_s, R_s) <- H^H A H
            sbr_two_sided<R, C, BMAX, G, P>(S, vc, tau, l, Hg, ldi, r, tid, g, s == 0 ? dd + j + 1 : nullptr);
            cur ^= 1;
            if (CL > 1) __threadfence(); else __threadfence_block();  // the step's writes, then its key
            gbar<G>(g);
            if (tid == 0) key[g] = (long long)j * KK + (s + 1 == nsteps ? KK - 1 : s + 1);
        }
    }
    // the partner may still read this CTA's keys and abort flag: leave together
    if (CL > 1) cluster.sync();
}

// ------------------------------------------------------------------ back-transform
// Window of the column in registers (FP32) -- one thread per column of Z (row-major, row stride n).
template <int BMAX>
__global__ void __launch_bounds__(128) k_sbr_bt_f32(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                   const double2* __restrict__ store_base,
                                                   const double* __restrict__ Yg, double* __restrict__ work) {
    __shared__ __align__(16) float2 vs[2][BMAX];
    __shared__ float2 ts[2];
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, b = d.band;
    const int c = blockIdx.x * 128 + threadIdx.x;
    if (blockIdx.x * 128 >= n) return;
    const bool act = c < n;
    const float2* V = reinterpret_cast<const float2*>(store_base + d.mat_off);
    const float2* T = V + sbr_nref(n, b) * b;
    const double* Y = Yg + d.sq_off;
    float2* Z = reinterpret_cast<float2*>(sbr_zbase(work, d));
    if (act) Z[c] = make_float2((float)Y[c], 0.f);  // row 0: no reflector touches it
    const int np = sbr_passes(n, b);
    float2 zr[BMAX];
    for (int s = 0; s < np; ++s) {
        const int jtop = n - 2 - s * b;
        const int64_t off = sbr_off(n, b, s);
        // window rows [r, r + BMAX), r = jtop + 1 + s b = n - 1
#pragma unroll
        for (int q = 0; q < BMAX; ++q) zr[q] = make_float2(0.f, 0.f);
        if (act) zr[0] = s == 0 ? make_float2((float)Y[(int64_t)(n - 1) * n + c], 0.f) : Z[(int64_t)(n - 1) * n + c];
        if (threadIdx.x < BMAX)
            vs[0][threadIdx.x] = threadIdx.x < b ? V[(off + jtop) * b + threadIdx.x] : make_float2(0.f, 0.f);
        if (threadIdx.x == 0) ts[0] = T[off + jtop];
        __syncthreads();
        int buf = 0;
#pragma unroll 1
        for (int j = jtop; j >= 0; --j) {
            float2 vn = make_float2(0.f, 0.f), tn = make_float2(0.f, 0.f);
            if (j > 0) {
                if (threadIdx.x < b) vn = V[(off + j - 1) * b + threadIdx.x];
                if (threadIdx.x == 0) tn = T[off + j - 1];
            }
            // w = v^H z, z -= tau w v; the dot product runs from the window's bottom up, so that
            // the row loaded last (zr[0]) is needed last
            float wr0 = 0.f, wi0 = 0.f, wr1 = 0.f, wi1 = 0.f;
#pragma unroll
            for (int q = BMAX - 2; q >= 0; q -= 2) {
                const float4 v2 = *reinterpret_cast<const float4*>(&vs[buf][q]);
                wr0 = fmaf(v2.x, zr[q].x, wr0);
                wr0 = fmaf(v2.y, zr[q].y, wr0);
                wi0 = fmaf(v2.x, zr[q].y, wi0);
                wi0 = fmaf(-v2.y, zr[q].x, wi0);
                wr1 = fmaf(v2.z, zr[q + 1].x, wr1);
                wr1 = fmaf(v2.w, zr[q + 1].y, wr1);
                wi1 = fmaf(v2.z, zr[q + 1].y, wi1);
                wi1 = fmaf(-v2.w, zr[q + 1].x, wi1);
            }
            const float2 t = ts[buf];
            const float wr = wr0 + wr1, wi = wi0 + wi1;
            // reload v from shared memory below rather than keep all of it in registers
            asm volatile("" ::: "memory");
            const float twr = t.x * wr - t.y * wi, twi = t.x * wi + t.y * wr;
            // (volatile: a second read of v, so that v need not stay in registers)
            const volatile float4* vv = reinterpret_cast<const volatile float4*>(&vs[buf][0]);
#pragma unroll
            for (int q = 0; q < BMAX; q += 2) {
                const float4 v2 = make_float4(vv[q / 2].x, vv[q / 2].y, vv[q / 2].z, vv[q / 2].w);
                zr[q].x = fmaf(-twr, v2.x, fmaf(twi, v2.y, zr[q].x));
                zr[q].y = fmaf(-twr, v2.y, fmaf(-twi, v2.x, zr[q].y));
                zr[q + 1].x = fmaf(-twr, v2.z, fmaf(twi, v2.w, zr[q + 1].x));
                zr[q + 1].y = fmaf(-twr, v2.w, fmaf(-twi, v2.z, zr[q + 1].y));
            }
            if (j > 0) {
                const int r = j + 1 + s * b;
                if (act && r + BMAX - 1 < n) Z[(int64_t)(r + BMAX - 1) * n + c] = zr[BMAX - 1];
#pragma unroll
                for (int q = BMAX - 1; q > 0; --q) zr[q] = zr[q - 1];
                if (act) {
                    const int64_t row = r - 1;
                    zr[0] = s == 0 ? make_float2((float)Y[row * n + c], 0.f) : Z[row * n + c];
                }
                if (threadIdx.x < BMAX) vs[buf ^ 1][threadIdx.x] = vn;
                if (threadIdx.x == 0) ts[buf ^ 1] = tn;
            }
            __syncthreads();
            buf ^= 1;
        }
        const int r0 = 1 + s * b;
        if (act) {
#pragma unroll
            for (int q = 0; q < BMAX; ++q)
                if (r0 + q < n) Z[(int64_t)(r0 + q) * n + c] = zr[q];
        }
    }
}

// FP64: the same with the window in shared memory (a column per thread, BMAX rows).
template <int BMAX>
__global__ void __launch_bounds__(128) k_sbr_bt_f64(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                   const double2* __restrict__ store_base,
                                                   const double* __restrict__ Yg, double* __restrict__ work) {
    extern __shared__ __align__(16) double2 sbt_smem[];
    double2* vs = sbt_smem;                 // [2][BMAX]
    double2* ts = vs + 2 * BMAX;            // [2]
    double2* win = ts + 2;                  // [BMAX][128]
    const MmfDesc d = descs[idx[blockIdx.y]];
    const int n = d.n, b = d.band;
    const int c = blockIdx.x * 128 + threadIdx.x;
    if (blockIdx.x * 128 >= n) return;
    const bool act = c < n;
    const double2* V = store_base + d.mat_off;
    const double2* T = V + sbr_nref(n, b) * b;
    const double* Y = Yg + d.sq_off;
    double2* Z = reinterpret_cast<double2*>(sbr_zbase(work, d));
    const int tx = threadIdx.x;
    if (act) Z[c] = make_double2(Y[c], 0.0);
    const int np = sbr_passes(n, b);
    for (int s = 0; s < np; ++s) {
        const int jtop = n - 2 - s * b;
        const int64_t off = sbr_off(n, b, s);
        int top = 0;  // window slot of the window's first row (circular)
        for (int q = 0; q < BMAX; ++q) win[q * 128 + tx] = make_double2(0.0, 0.0);
        if (act) win[tx] = s == 0 ? make_double2(Y[(int64_t)(n - 1) * n + c], 0.0) : Z[(int64_t)(n - 1) * n + c];
        if (tx < BMAX) vs[tx] = tx < b ? V[(off + jtop) * b + tx] : make_double2(0.0, 0.0);
        if (tx == 0) ts[0] = T[off + jtop];
        __syncthreads();
        int buf = 0;
        for (int j = jtop; j >= 0; --j) {
            double2 vn = make_double2(0.0, 0.0), tn = make_double2(0.0, 0.0);
            if (j > 0) {
                if (tx < b) vn = V[(off + j - 1) * b + tx];
                if (tx == 0) tn = T[off + j - 1];
            }
            const double2* vv = vs + buf * BMAX;
            double2 w = make_double2(0.0, 0.0);
            for (int q = 0; q < BMAX; ++q) w = w + cmulc(vv[q], win[((top + q) % BMAX) * 128 + tx]);
            const double2 tw = ts[buf] * w;
            for (int q = 0; q < BMAX; ++q) {
                double2& z = win[((top + q) % BMAX) * 128 + tx];
                z = z - tw * vv[q];
            }
            if (j > 0) {
                const int r = j + 1 + s * b;
                const int bot = (top + BMAX - 1) % BMAX;
                if (act && r + BMAX - 1 < n) Z[(int64_t)(r + BMAX - 1) * n + c] = win[bot * 128 + tx];
                top = bot;  // the slot of the leaving row takes the new first row
                const int64_t row = r - 1;
                win[top * 128 + tx] = act ? (s == 0 ? make_double2(Y[row * n + c], 0.0) : Z[row * n + c])
                                          : make_double2(0.0, 0.0);
                if (tx < BMAX) vs[(buf ^ 1) * BMAX + tx] = vn;
                if (tx == 0) ts[buf ^ 1] = tn;
            }
            __syncthreads();
            buf ^= 1;
        }
        const int r0 = 1 + s * b;
        if (act)
            for (int q = 0; q < BMAX; ++q)
                if (r0 + q < n) Z[(int64_t)(r0 + q) * n + c] = win[((top + q) % BMAX) * 128 + tx];
        __syncthreads();
    }
}

// Z (row-major, work slot) -> the back-transform's output (column-major, ld; FP32 for the mixed
// path, FP64 otherwise), 32 x 32 tiles through shared memory.
template <class R>
__global__ void __launch_bounds__(256) k_sbr_out(const MmfDesc* __restrict__ descs, const int* __restrict__ idx,
                                                const double* __restrict__ work, typename Cx<R>::T* __restrict__ out) {
    typedef typename Cx<R>::T C;
    __shared__ C tile[32][33];
    const MmfDesc d = descs[idx[blockIdx.z]];
    const int n = d.n;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    if (r0 >= n || c0 >= n) return;
    const C* Z = reinterpret_cast<const C*>(sbr_zbase(const_cast<double*>(work), d));
    C* O = out + d.mat_off;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int q = ty; q < 32; q += 8) {
        const int r = r0 + q, c = c0 + tx;
        if (r < n && c < n) tile[q][tx] = Z[(int64_t)r * n + c];
    }
    __syncthreads();
    for (int q = ty; q < 32; q += 8) {
        const int c = c0 + q, r = r0 + tx;
        if (r < n && c < n) O[(int64_t)c * d.ld + r] = tile[tx][q];
    }
}

// ------------------------------------------------------------------ launchers
template <class R, int BMAX, int G, int NG, int CL>
static cudaError_t launch_chase(const MmfLaunch& L, void* H, double2* store, double* dvec, double* evec,
                                int* status) {
    typedef typename Cx<R>::T C;
    static_assert(sizeof(SbrGroup<C, BMAX, G / BMAX>) % 16 == 0, "group blocks keep 16-byte alignment");
    const size_t sm = sbr_hdr(NG) + sizeof(SbrGroup<C, BMAX, G / BMAX>) * NG;
    cudaError_t e = cudaFuncSetAttribute(k_sbr_chase<R, BMAX, G, NG, CL>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(L.count * CL);
    cfg.blockDim = dim3(G * NG);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = L.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_sbr_chase<R, BMAX, G, NG, CL>, L.desc, L.idx, (C*)H, (C*)store, dvec, evec,
                              status);
}

template <int BMAX>
static cudaError_t launch_bt(const MmfLaunch& L, const double2* store, const double* Y, double* work, int fp32) {
    dim3 g((L.nmax + 127) / 128, L.count);
    if (fp32) {
        k_sbr_bt_f32<BMAX><<<g, 128, 0, L.stream>>>(L.desc, L.idx, store, Y, work);
    } else {
        const size_t sm = sizeof(double2) * (2 * BMAX + 2 + (size_t)BMAX * 128);
        cudaError_t e = cudaFuncSetAttribute(k_sbr_bt_f64<BMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_sbr_bt_f64<BMAX><<<g, 128, sm, L.stream>>>(L.desc, L.idx, store, Y, work);
    }
    return cudaGetLastError();
}

// The paired (two-SM) chase can be switched off for comparison: MMF_SBR_PAIRS=0 in the
// environment.
static bool sbr_pairs_enabled() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("MMF_SBR_PAIRS");
        v = (e && e[0] == '0') ? 0 : 1;
    }
    return v == 1;
}

int mmf_sbr_class(int b) { return b <= 8 ? 8 : b <= 16 ? 16 : b <= 32 ? 32 : b <= 64 ? 64 : 0; }

cudaError_t mmf_launch_sbr_chase(const MmfLaunch& L, int bmax, void* H, double2* store, double* dvec, double* evec,
                                 int* status, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    // two CTAs (SMs) per system for the widest band while the pairs fit the GPU in one wave
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const bool pair = sbr_pairs_enabled() && 2 * L.count <= sms;
    if (fp32) {
        switch (bmax) {
            case 8: return launch_chase<float, 8, 32, 15, 1>(L, H, store, dvec, evec, status);
            case 16: return launch_chase<float, 16, 32, 15, 1>(L, H, store, dvec, evec, status);
            case 32: return launch_chase<float, 32, 64, 8, 1>(L, H, store, dvec, evec, status);
            case 64:
                return pair ? launch_chase<float, 64, 128, 3, 2>(L, H, store, dvec, evec, status)
                            : launch_chase<float, 64, 128, 3, 1>(L, H, store, dvec, evec, status);
        }
    } else {
        switch (bmax) {
            case 8: return launch_chase<double, 8, 32, 15, 1>(L, H, store, dvec, evec, status);
            case 16: return launch_chase<double, 16, 32, 12, 1>(L, H, store, dvec, evec, status);
            case 32: return launch_chase<double, 32, 64, 4, 1>(L, H, store, dvec, evec, status);
            case 64:
                return pair ? launch_chase<double, 64, 128, 1, 2>(L, H, store, dvec, evec, status)
                            : launch_chase<double, 64, 128, 1, 1>(L, H, store, dvec, evec, status);
        }
    }
    return cudaErrorInvalidValue;
}

cudaError_t mmf_launch_sbr_out(const MmfLaunch& L, double* work, float2* Zout) {
    if (L.count <= 0) return cudaSuccess;
    const int t = (L.nmax + 31) / 32;
    k_sbr_out<float><<<dim3(t, t, L.count), 256, 0, L.stream>>>(L.desc, L.idx, work, Zout);
    return cudaGetLastError();
}

cudaError_t mmf_launch_sbr_bt(const MmfLaunch& L, int bmax, const double2* store, const double* Y, double* work,
                              void* Zout, int fp32) {
    if (L.count <= 0) return cudaSuccess;
    cudaError_t e;
    switch (bmax) {
        case 8: e = launch_bt<8>(L, store, Y, work, fp32); break;
        case 16: e = launch_bt<16>(L, store, Y, work, fp32); break;
        case 32: e = launch_bt<32>(L, store, Y, work, fp32); break;
        case 64: e = launch_bt<64>(L, store, Y, work, fp32); break;
        default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    const int t = (L.nmax + 31) / 32;
    dim3 g(t, t, L.count);
    if (fp32) k_sbr_out<float><<<g, 256, 0, L.stream>>>(L.desc, L.idx, work, (float2*)Zout);
    else k_sbr_out<double><<<g, 256, 0, L.stream>>>(L.desc, L.idx, work, (double2*)Zout);
    return cudaGetLastError();
}
