// fr_p1.cu -- kernels of the free-cost parametrisation (Problem (8): one cost c_uik per cell).
//
// One persistent CTA processes consumers u = blockIdx.x, blockIdx.x + G, ... (Algorithm 1's
// parallel loop over consumers). A thread owns R consecutive items (rows) of the consumer; their
// costs stay in registers for the whole Sinkhorn solve, so the L iterations touch HBM only once.
//
// Sinkhorn (Problem (7)) runs in the fused single-pass log-domain form, in log2 units
// c' = c / (eps ln 2), g' = g / (eps ln 2):
//   p_ik = 2^(g'_k - c~_ik),  S_i = sum_k p_ik,  x_ik = p_ik / S_i       (row update, Eq. 1)
//   cs_k = sum_i x_ik,        g'_k += log2 b_k - log2 cs_k               (column update, Eq. 2)
// which equals the textbook two-pass update (f_i = -eps LSE_k, g_k = eps log b_k - eps LSE_i)
// algebraically and costs one exp2 per cell per iteration. c~_ik = c'_ik + shift_i carries a
// per-row shift fixed at the start of the solve (row max), so 2^(.) stays in range without a
// max pass per iteration; a row whose S_i leaves [2^-64, 2^64] is re-shifted exactly.
//
// The last iteration emits x (the policy right after the last row update, rows sum to 1) and adds
// r(u,i) * sum_{k<K} e_k x_ik into per-thread impact accumulators (Eq. 4) that persist over the
// CTA's consumers; they are written once per launch to part[blockIdx][i] and combined across CTAs
// by the reduction kernel in a fixed order.
//
// MODE_UPDATE_SWEEP first takes the gradient step of Algorithm 1 for the consumer: it re-forms
// the previous policy from C and g^(L-1), computes dF/dC by implicit differentiation of the
// optimality conditions of Problem (7),
//   h_i = sum_k x_ik G_ik, q_k = sum_i x_ik G_ik, (diag(cs) - X^T X) beta = q - X^T h (beta_last = 0),
//   alpha_i = h_i - sum_k x_ik beta_k,  dF/dc_ik = -(1/eps) x_ik (G_ik - alpha_i - beta_k),
// with G_ik = r(u,i) e_k / Imp_i, applies Adam (ascent) to C in registers, writes C and the
// moments back, and then solves Sinkhorn on the new costs without reloading them.
#include "fr_device.cuh"
#include "fr_internal.h"

namespace fr {

namespace {

// dynamic shared-memory layout (floats unless noted)
struct Smem {
    float* g;     // [NCP] current g'
    float* gp;    // [NCP] g^(L-1)' of the previous solve (update mode)
    float* l2b;   // [NCP] log2 b
    float* e;     // [NCP] exposure
    float* red;   // [W][3][P] reduction scratch
    float* out;   // [3][NCP] reduction results
    float* beta;  // [NCP]
    double* A;    // [n*n] Gram system (update mode)
    double* rhs;  // [NCP]
    float* X;     // [nc][ld] policy of the consumer (update mode)
};

constexpr int NCP_ALIGN = 4;

__host__ __device__ inline int ncp_of(int nc) { return (nc + NCP_ALIGN - 1) / NCP_ALIGN * NCP_ALIGN; }

__host__ __device__ inline size_t smem_layout(int nc, int ld, int W, int P, int mode, Smem* s,
                                              unsigned char* base) {
    const int ncp = ncp_of(nc);
    const int n = nc - 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += (bytes + 15) / 16 * 16;
        return o;
    };
    size_t o_g = take(sizeof(float) * ncp), o_gp = take(sizeof(float) * ncp);
    size_t o_l2b = take(sizeof(float) * ncp), o_e = take(sizeof(float) * ncp);
    size_t o_red = take(sizeof(float) * (size_t)W * 3 * P);
    size_t o_out = take(sizeof(float) * 3 * ncp);
    size_t o_beta = take(sizeof(float) * ncp);
    size_t o_A = 0, o_rhs = 0, o_X = 0;
    if (mode != MODE_SWEEP) {
        o_A = take(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
        o_rhs = take(sizeof(double) * ncp);
        o_X = take(sizeof(float) * (size_t)nc * ld);
    }
    if (s) {
        s->g = (float*)(base + o_g);
        s->gp = (float*)(base + o_gp);
        s->l2b = (float*)(base + o_l2b);
        s->e = (float*)(base + o_e);
        s->red = (float*)(base + o_red);
        s->out = (float*)(base + o_out);
        s->beta = (float*)(base + o_beta);
        s->A = (double*)(base + o_A);
        s->rhs = (double*)(base + o_rhs);
        s->X = (float*)(base + o_X);
    }
    return off;
}

// Cholesky solve of the n x n SPD system in s.A (row-major, lower triangle used) with right-hand
// side s.rhs, by one warp, in double precision. Pivots below `floor` are raised to it (a column
// with no mass leaves the Laplacian-like Gram matrix singular; its beta is then ~0).
__device__ void warp_cholesky_solve(double* A, double* rhs, int n, int lane) {
    double dmax = 0.0;
    for (int j = 0; j < n; ++j) dmax = fmax(dmax, A[j * n + j]);
    const double floor_ = 1e-13 * fmax(dmax, 1e-300);
    for (int j = 0; j < n; ++j) {
        __syncwarp();
        const double ljj = sqrt(fmax(A[j * n + j], floor_));
        for (int i = j + 1 + lane; i < n; i += 32) A[i * n + j] /= ljj;
        __syncwarp();
        if (lane == 0) A[j * n + j] = ljj;
        const int m = n - j - 1;
        for (int idx = lane; idx < m * m; idx += 32) {
            const int i = j + 1 + idx / m, k = j + 1 + idx % m;
            if (k <= i) A[i * n + k] -= A[i * n + j] * A[k * n + j];
        }
    }
    __syncwarp();
    for (int j = 0; j < n; ++j) {  // L y = rhs
        const double yj = rhs[j] / A[j * n + j];
        __syncwarp();
        for (int i = j + 1 + lane; i < n; i += 32) rhs[i] -= A[i * n + j] * yj;
        if (lane == 0) rhs[j] = yj;
        __syncwarp();
    }
    for (int j = n - 1; j >= 0; --j) {  // L^T z = y
        const double zj = rhs[j] / A[j * n + j];
        __syncwarp();
        for (int i = lane; i < j; i += 32) rhs[i] -= A[j * n + i] * zj;
        if (lane == 0) rhs[j] = zj;
        __syncwarp();
    }
}

template <int NCB, int R, bool EXACT, int MODE>
__global__ void __launch_bounds__(512) p1_kernel(const P1Args a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int P = pow2ceil(NCB);
    const int nc = EXACT ? NCB : a.nc;
    const int ncp = ncp_of(nc);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, W = blockDim.x >> 5;
    const int I = a.I, ld = a.ld;
    const int i0 = tid * R;
    const bool any_row = i0 < I;
    Smem s;
    smem_layout(nc, ld, W, P, MODE, &s, smem_raw);

    if (a.st->stop) return;  // fr_solve reached its threshold: the remaining steps are no-ops

    for (int k = tid; k < ncp; k += blockDim.x) {
        s.l2b[k] = k < nc ? a.log2b[k] : 0.f;
        s.e[k] = k < nc ? a.e[k] : 0.f;
    }

    float acc_imp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc_imp[r] = 0.f;
    double gn2 = 0.0;

    // Adam bias corrections for this step (t counts applied steps before this one)
    float step_size = a.lr, bc2s = 1.f;
    if (MODE == MODE_UPDATE_SWEEP && a.optimizer == 0) {
        const double t1 = (double)(a.st->t + 1);
        const double bc1 = 1.0 - pow((double)a.beta1, t1);
        const double bc2 = 1.0 - pow((double)a.beta2, t1);
        step_size = (float)((double)a.lr / bc1);
        bc2s = (float)sqrt(bc2);
    }

    for (int u = blockIdx.x; u < a.U; u += gridDim.x) {
        const size_t tile = (size_t)u * nc * ld;
        if (tid < nc) {
            s.g[tid] = a.warm ? a.gL[(size_t)u * nc + tid] : 0.f;
            if (MODE != MODE_SWEEP) s.gp[tid] = a.gP[(size_t)u * nc + tid];
        }
        float rr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) rr[r] = 0.f;
        if (any_row) ldv<R>(rr, a.r + (size_t)u * ld + i0);
        bool vr[R];
#pragma unroll
        for (int r = 0; r < R; ++r) vr[r] = i0 + r < I;

        // costs of the owned rows, natural units
        float c[R][NCB];
#pragma unroll
        for (int k = 0; k < NCB; ++k) {
            float tmp[R];
            if ((EXACT || k < nc) && any_row) {
                ldv<R>(tmp, a.C + tile + (size_t)k * ld + i0);
            } else {
#pragma unroll
                for (int r = 0; r < R; ++r) tmp[r] = 0.f;
            }
#pragma unroll
            for (int r = 0; r < R; ++r) c[r][k] = tmp[r];
        }
        __syncthreads();  // s.g / s.gp / s.e / s.l2b visible

        if constexpr (MODE != MODE_SWEEP) {
            // ---------------- gradient of F at the previous policy ------------------------------
            float wr[R], om[R];
#pragma unroll
            for (int r = 0; r < R; ++r) om[r] = 0.f;
            if (any_row) ldv<R>(om, a.omega + i0);
#pragma unroll
            for (int r = 0; r < R; ++r) wr[r] = vr[r] ? om[r] * rr[r] : 0.f;  // dF/dx_ik = wr_i e_k
            float acc[3][NCB];  // q, cs, X^T h partials
#pragma unroll
            for (int k = 0; k < NCB; ++k) acc[0][k] = acc[1][k] = acc[2][k] = 0.f;
            float hrow[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                hrow[r] = 0.f;
                if (!vr[r]) continue;
                float p[NCB];
                float M = -INFINITY;
#pragma unroll
                for (int k = 0; k < NCB; ++k)
                    if (EXACT || k < nc) M = fmaxf(M, s.gp[k] - c[r][k] * a.inv_eps_ln2);
                float S = 0.f;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    p[k] = (EXACT || k < nc) ? ex2(s.gp[k] - c[r][k] * a.inv_eps_ln2 - M) : 0.f;
                    S += p[k];
                }
                const float inv = 1.f / S;
                float h = 0.f;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    p[k] *= inv;
                    if (EXACT || k < nc) h += p[k] * (wr[r] * s.e[k]);
                }
                hrow[r] = h;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    if (EXACT || k < nc) {
                        s.X[k * ld + i0 + r] = p[k];
                        acc[0][k] += p[k] * (wr[r] * s.e[k]);
                        acc[1][k] += p[k];
                        acc[2][k] += p[k] * h;
                    }
                }
            }
            cta_reduce<NCB, 3>(acc, nc, s.red, s.out, ncp);  // s.out: [q | cs | X^T h]
            // Gram block M[0:n,0:n] of diag(cs) - X^T X (rows of x sum to 1, so the diagonal is
            // sum_i x_ik (1 - x_ik) without cancellation), and the right-hand side q - X^T h.
            const int n = nc - 1;
            const int npairs = n * (n + 1) / 2;
            for (int pidx = warp; pidx < npairs; pidx += W) {
                int k = 0, rem = pidx;
                while (rem >= n - k) { rem -= n - k; ++k; }
                const int l = k + rem;
                const float* xk = s.X + k * ld;
                const float* xl = s.X + l * ld;
                float sum = 0.f;
                if (k == l) {
                    for (int i = lane; i < I; i += 32) sum += xk[i] * (1.f - xk[i]);
                } else {
                    for (int i = lane; i < I; i += 32) sum -= xk[i] * xl[i];
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(FULL, sum, o);
                if (lane == 0) {
                    s.A[k * n + l] = (double)sum;
                    s.A[l * n + k] = (double)sum;
                }
            }
            for (int k = tid; k < n; k += blockDim.x)
                s.rhs[k] = (double)s.out[k] - (double)s.out[2 * ncp + k];
            __syncthreads();
            if (warp == 0) warp_cholesky_solve(s.A, s.rhs, n, lane);
            __syncthreads();
            for (int k = tid; k < ncp; k += blockDim.x) s.beta[k] = k < n ? (float)s.rhs[k] : 0.f;
            __syncthreads();

            float alpha[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float sb = 0.f;
                if (vr[r]) {
#pragma unroll
                    for (int k = 0; k < NCB; ++k)
                        if (EXACT || k < nc) sb += s.X[k * ld + i0 + r] * s.beta[k];
                }
                alpha[r] = hrow[r] - sb;
            }
            float gsq = 0.f;
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                if (!(EXACT || k < nc) || !any_row) continue;
                float xk[R], gr[R];
                ldv<R>(xk, s.X + k * ld + i0);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    gr[r] = vr[r] ? -a.inv_eps * xk[r] * (wr[r] * s.e[k] - alpha[r] - s.beta[k]) : 0.f;
                    gsq += gr[r] * gr[r];
                }
                if constexpr (MODE == MODE_GRAD) {
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        if (vr[r]) a.dC[((size_t)u * I + i0 + r) * nc + k] = gr[r];
                } else {
                    const size_t off = tile + (size_t)k * ld + i0;
                    if (a.optimizer == 1) {
#pragma unroll
                        for (int r = 0; r < R; ++r) c[r][k] += a.lr * gr[r];
                    } else {
                        float mm[R], vv[R];
                        ldv<R>(mm, a.m1 + off);
                        ldv<R>(vv, a.m2 + off);
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            mm[r] = a.beta1 * mm[r] + (1.f - a.beta1) * gr[r];
                            vv[r] = a.beta2 * vv[r] + (1.f - a.beta2) * gr[r] * gr[r];
                            c[r][k] += step_size * mm[r] / (sqrtf(vv[r]) / bc2s + a.adam_eps);
                        }
                        stv<R>(a.m1 + off, mm);
                        stv<R>(a.m2 + off, vv);
                    }
                    float cw[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) cw[r] = c[r][k];
                    stv<R>(a.C + off, cw);
                }
            }
            gn2 += (double)gsq;
            if constexpr (MODE == MODE_GRAD) {
                if (a.dr) {
                    // dF/dr(u,i) = (dF/dImp_i) sum_{k<K} e_k x_ik (C does not depend on r)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (!vr[r]) continue;
                        float v = 0.f;
#pragma unroll
                        for (int k = 0; k < NCB; ++k)
                            if ((EXACT || k < nc) && k < a.K) v += s.e[k] * s.X[k * ld + i0 + r];
                        a.dr[(size_t)u * I + i0 + r] = om[r] * v;
                    }
                }
                __syncthreads();
                continue;  // no solve in gradient mode
            }
            __syncthreads();  // s.X / s.beta reused by the next consumer
        }

        // ---------------- Sinkhorn solve on the consumer's (new) costs ----------------------------
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float M = -INFINITY;
#pragma unroll
            for (int k = 0; k < NCB; ++k) {
                if (EXACT || k < nc) {
                    c[r][k] *= a.inv_eps_ln2;
                    M = fmaxf(M, s.g[k] - c[r][k]);
                } else {
                    c[r][k] = INFINITY;  // padding column: 2^(-inf) = 0
                }
            }
#pragma unroll
            for (int k = 0; k < NCB; ++k)
                if (EXACT || k < nc) c[r][k] += vr[r] ? M : 0.f;
        }
        for (int l = 0; l < a.L; ++l) {
            const bool last = l == a.L - 1;
            if (last && tid < nc) a.gP[(size_t)u * nc + tid] = s.g[tid];
            float gk[NCB];
#pragma unroll
            for (int k = 0; k < NCB; ++k) gk[k] = (EXACT || k < nc) ? s.g[k] : 0.f;
            float cs[1][NCB];
#pragma unroll
            for (int k = 0; k < NCB; ++k) cs[0][k] = 0.f;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if (!vr[r]) continue;
                float p[NCB];
                float S = 0.f;
#pragma unroll
                for (int k = 0; k < NCB; ++k) {
                    p[k] = ex2(gk[k] - c[r][k]);
                    S += p[k];
                }
                if (!(S >= 0x1p-64f && S <= 0x1p64f)) {  // re-shift this row exactly
                    float M = -INFINITY;
#pragma unroll
                    for (int k = 0; k < NCB; ++k)
                        if (EXACT || k < nc) M = fmaxf(M, gk[k] - c[r][k]);
                    S = 0.f;
#pragma unroll
                    for (int k = 0; k < NCB; ++k) {
                        if (EXACT || k < nc) c[r][k] += M;
                        p[k] = ex2(gk[k] - c[r][k]);
                        S += p[k];
                    }
                }
                const float inv = rcp_approx(S);
#pragma unroll
                for (int k = 0; k < NCB; ++k) cs[0][k] += p[k] * inv;
                if (last) {
                    float v = 0.f;
#pragma unroll
                    for (int k = 0; k < NCB; ++k)
                        if (k < a.K) v += s.e[k] * p[k];
                    acc_imp[r] += rr[r] * (v * inv);
                }
            }
            cta_reduce<NCB, 1>(cs, nc, s.red, s.out, ncp);
            if (tid < nc) s.g[tid] += s.l2b[tid] - log2f(fmaxf(s.out[tid], 1e-37f));
            __syncthreads();
        }
        if (tid < nc) a.gL[(size_t)u * nc + tid] = s.g[tid];
        __syncthreads();
    }

    if constexpr (MODE != MODE_GRAD) {
        if (i0 < ld) stv<R>(a.part + (size_t)blockIdx.x * ld + i0, acc_imp);
    }
    if constexpr (MODE == MODE_UPDATE_SWEEP) {
        // CTA sum of the squared gradient in double, fixed order
        double* s_d = reinterpret_cast<double*>(s.red);
        __syncthreads();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) gn2 += __shfl_xor_sync(FULL, gn2, o);
        if (lane == 0) s_d[warp] = gn2;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < W; ++w) t += s_d[w];
            a.gn2_part[blockIdx.x] = t;
        }
    }
}

template <int NCB, int R, bool EXACT>
P1Variant make_variant(int threads) {
    P1Variant v;
    v.ncb = NCB;
    v.rows = R;
    v.exact = EXACT;
    v.threads = threads;
    v.smem = 0;
    v.fn[MODE_SWEEP] = (const void*)p1_kernel<NCB, R, EXACT, MODE_SWEEP>;
    v.fn[MODE_UPDATE_SWEEP] = (const void*)p1_kernel<NCB, R, EXACT, MODE_UPDATE_SWEEP>;
    v.fn[MODE_GRAD] = (const void*)p1_kernel<NCB, R, EXACT, MODE_GRAD>;
    return v;
}

}  // namespace

size_t p1_smem_bytes(const P1Variant& v, int mode, int nc, int ld) {
    return smem_layout(nc, ld, v.threads / 32, pow2ceil(v.ncb), mode, nullptr, nullptr);
}

// Compiled variants: exact column counts for the hot shapes, padded buckets for the rest.
bool p1_select(int nc, int I, P1Variant* out) {
    // CTA size: one thread per R items, at most 512 threads (the kernels' launch bound)
    auto threads_for = [&](int R) {
        int t = (I + R - 1) / R;
        return (t + 31) / 32 * 32;
    };
    P1Variant v;
    if (nc == 11 && threads_for(4) <= 512) {
        v = make_variant<11, 4, true>(threads_for(4));
    } else if (nc == 50 && threads_for(1) <= 512) {
        v = make_variant<50, 1, true>(threads_for(1));
    } else if (nc <= 8 && threads_for(4) <= 512) {
        v = make_variant<8, 4, false>(threads_for(4));
    } else if (nc <= 16 && threads_for(4) <= 512) {
        v = make_variant<16, 4, false>(threads_for(4));
    } else if (nc <= 32 && threads_for(2) <= 512) {
        v = make_variant<32, 2, false>(threads_for(2));
    } else if (nc <= 64 && threads_for(1) <= 512) {
        v = make_variant<64, 1, false>(threads_for(1));
    } else {
        return false;
    }
    *out = v;
    return true;
}

cudaError_t p1_launch(const P1Variant& v, int mode, const P1Args& a, cudaStream_t s) {
    const size_t smem = p1_smem_bytes(v, mode, a.nc, a.ld);
    void* args[] = {const_cast<P1Args*>(&a)};
    return cudaLaunchKernel(v.fn[mode], dim3(a.G), dim3(v.threads), args, smem, s);
}

}  // namespace fr
