// CLOMP fit with the image priors: the total variation of an image (Eq. 6)
// and the local variation (Eq. 7).  The batch is a sequence of images of W
// consecutive columns, column j of an image being the signal x_j = D s_j
// (H = N pixels).
//
// Total variation.  Its vertical part is the 1-D form of Eq. 5 per column
// and already sits in A^T A (k_prior.cu), so it reaches the per-signal Gram
// matrices G = A_S^T A_S + (2w/H)(Delta D_S)^T(Delta D_S).  Its horizontal
// part, (w/W) sum_j ||x_j - x_{j+1}||^2, couples neighbouring columns; for a
// basis with orthonormal columns (D^T D = I: the DCT, or no basis) it equals
// (w/W) sum_j ||s_j - s_{j+1}||^2, whose gradient with respect to column j's
// support coefficients is
//   (2w/W) (c_j s_j - s_{j-1}|_{S_j} - s_{j+1}|_{S_j}),
// c_j the number of neighbours (1 at the image's edges, else 2) and
// s_{j+-1}|_{S_j} the neighbour's coefficients at the atoms of S_j (zero where
// the neighbour has not selected the atom).
//
// Local variation.  LV(I) = (1/B) sum_b sigma_b over the 3 x 3 windows b at
// every placement (B = (H-2)(W-2)), sigma_b the sample standard deviation of
// the window's nine pixels; dLV/dI_p = (1/B) sum_{b containing p} (I_p -
// mu_b) / (8 sigma_b) (0 for a constant window; sigma_b smoothed as
// sqrt(var + eps^2) when eps > 0), taken back to the support
// coefficients by D_S^T.  It is not quadratic, so every step synthesises the
// pixel columns x_j = D_S s_j, forms the windows' means and deviations, and
// back-projects the pixel gradient (any basis D).
//
// The columns of an image take their Adam steps together, each step's
// gradients from the coefficients before it, so an image is one thread-block
// cluster: one warp per column, lane q owning coordinate q (row q of G in
// registers).  Every step the columns publish their coefficients (and, with
// LV, their pixels and then their windows' statistics) in shared memory;
// cluster barriers order publication and reads, and columns at a CTA edge
// read their neighbours through distributed shared memory.  Stopped columns
// keep their coefficients and still serve as neighbours.
#include <cooperative_groups.h>

#include "k_fit.cuh"

namespace cg = cooperative_groups;

namespace cs {
namespace {

constexpr int kImgWarps = 32;   // columns (warps) per CTA at most
constexpr int kLvMaxN = 256;    // pixels per column with the local variation

struct ImgArgs {
    int W, wpc;          // image width; columns per CTA
    float lam_h;         // 2 w_tv / W (0: no horizontal term)
    float lv_scale;      // w_lv / ((H - 2)(W - 2)) (0: no local variation)
    float lv_eps2;       // the window deviation's smoothing, squared
    const float* D;      // H x n basis (column-major, leading dimension ldd), nullptr: x = s
    int H, ldd, NP;      // pixels per column, D's leading dimension, H rounded up to 32
};

// Shared-memory address of column `cc` (of this image) in the CTA that owns
// it: `base` is this CTA's copy of a per-column array with `stride` elements
// per column.
template <class T>
__device__ __forceinline__ T* column_slot(cg::cluster_group& cl, T* base, int stride, int cc, int wpc, int rank) {
    const int r = cc / wpc;
    T* local = base + (size_t)(cc - r * wpc) * stride;
    return r == rank ? local : cl.map_shared_rank(local, r);
}

template <int KT, bool LV>
__global__ void __launch_bounds__(1024, 1) k_clfit_image(IterArgs a, ClArgs c, ImgArgs g) {
    static_assert(KT % 8 == 0 && KT >= 8 && KT <= 32, "one coordinate per lane");
    constexpr int NR = kLvMaxN / 32;
    cg::cluster_group cl = cg::this_cluster();
    __shared__ __align__(16) float sh_s[2][kImgWarps][KT];
    __shared__ int sh_off[kImgWarps][KT];      // LV: column offsets of the support atoms in D
    __shared__ float2 sh_tab[kAdamStaged];
    extern __shared__ __align__(16) float dyn[];   // LV: pixels [wpc][NP], then window stats [wpc][NP]
    const float2* tab = stage_adam(c, sh_tab);

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
    const int W = g.W, wpc = g.wpc;
    const int img = blockIdx.x / csz;
    const int col = rank * wpc + w;                 // column within the image
    const bool in_img = col < W;
    const int b = img * W + (in_img ? col : 0);
    const int K = a.kmax;
    const bool live = in_img && a.status[b] < 0;
    // support size: a live column got this iteration's atom from the selection
    const int sz = in_img ? a.n_iter[b] + (live ? 1 : 0) : 0;
    const bool on = lane < sz;

    // row q of G: in registers, or (LV, whose pixel work needs the registers)
    // read from L1 every step
    constexpr int GR = LV ? 1 : KT;
    float grow[GR];
    const float* Gr = a.G + ((size_t)b * K + (on ? lane : 0)) * K;
    if constexpr (!LV) {
#pragma unroll
        for (int p = 0; p < KT; ++p) grow[p] = (live && on && p < sz) ? Gr[p] : 0.f;
    }
    float s = on ? a.coef[(size_t)b * a.k + lane] : 0.f;
    float mo = (live && on && !c.reset) ? a.am[(size_t)b * K + lane] : 0.f;
    float ve = (live && on && !c.reset) ? a.av[(size_t)b * K + lane] : 0.f;
    const float bb = (live && on) ? a.bvec[(size_t)b * K + lane] : 0.f;

    // where this lane's atom sits in the neighbours' supports (-1: absent)
    const int atom = on ? a.support[(size_t)b * a.k + lane] : -1;
    int pos_l = -1, pos_r = -1;
    if (live && on && g.lam_h != 0.f) {
        if (col > 0) {
            const int nb = b - 1;
            const int nsz = a.n_iter[nb] + (a.status[nb] < 0 ? 1 : 0);
            for (int p = 0; p < nsz; ++p)
                if (a.support[(size_t)nb * a.k + p] == atom) pos_l = p;
        }
        if (col < W - 1) {
            const int nb = b + 1;
            const int nsz = a.n_iter[nb] + (a.status[nb] < 0 ? 1 : 0);
            for (int p = 0; p < nsz; ++p)
                if (a.support[(size_t)nb * a.k + p] == atom) pos_r = p;
        }
    }
    const float c_self = g.lam_h * (float)((col > 0 ? 1 : 0) + (col < W - 1 ? 1 : 0));
    // neighbours' coefficient slots: the next warp of this CTA, or the edge
    // warp of the neighbouring CTA of the cluster
    const bool l_remote = w == 0, r_remote = w == wpc - 1;

    // local variation: this column's pixels and window statistics, the next
    // two columns' pixels (windows whose left column is this one) and the
    // previous two columns' statistics (windows that contain this column)
    float* xs = dyn;
    float2* st = reinterpret_cast<float2*>(dyn + (size_t)wpc * g.NP);
    float* my_x = xs + (size_t)w * g.NP;
    float2* my_st = st + (size_t)w * g.NP;
    if (LV) {
        if (lane < KT) sh_off[w][lane] = (on && g.D) ? atom * g.ldd : (on ? atom : 0);
    }
    __syncthreads();
    const bool lv_left = LV && in_img && col + 2 < W;   // this column starts windows
    const float* x1 = nullptr;
    const float* x2 = nullptr;
    const float2* sm1 = nullptr;
    const float2* sm2 = nullptr;
    if (LV) {
        if (lv_left) {
            x1 = column_slot(cl, xs, g.NP, col + 1, wpc, rank);
            x2 = column_slot(cl, xs, g.NP, col + 2, wpc, rank);
        }
        if (in_img && col >= 1 && col - 1 + 2 < W) sm1 = column_slot(cl, st, g.NP, col - 1, wpc, rank);
        if (in_img && col >= 2) sm2 = column_slot(cl, st, g.NP, col - 2, wpc, rank);
    }
    const bool lv_self = LV && lv_left;   // windows starting at this column contain it too
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;

    for (int step = 0; step < c.steps; ++step) {
        const int par = step & 1;
        float* mine = sh_s[par][w];
        if (lane < KT) mine[lane] = s;
        if (LV) {
            __syncwarp();
            // x = D_S s (or s placed at its atoms)
            if (g.D) {
                float acc[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) acc[r] = 0.f;
                int q = 0;
                // four atoms at a time: 4 * NR independent loads in flight
                for (; q + 4 <= sz; q += 4) {
                    const float* d0 = g.D + sh_off[w][q];
                    const float* d1 = g.D + sh_off[w][q + 1];
                    const float* d2 = g.D + sh_off[w][q + 2];
                    const float* d3 = g.D + sh_off[w][q + 3];
                    const float s0 = mine[q], s1 = mine[q + 1], s2 = mine[q + 2], s3 = mine[q + 3];
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = lane + 32 * r;
                        if (i < g.H) {
                            const float v0 = d0[i], v1 = d1[i], v2 = d2[i], v3 = d3[i];
                            acc[r] = fmaf(v3, s3, fmaf(v2, s2, fmaf(v1, s1, fmaf(v0, s0, acc[r]))));
                        }
                    }
                }
                for (; q < sz; ++q) {
                    const float sq = mine[q];
                    const float* dq = g.D + sh_off[w][q];
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = lane + 32 * r;
                        if (i < g.H) acc[r] = fmaf(dq[i], sq, acc[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (lane + 32 * r < g.NP) my_x[lane + 32 * r] = acc[r];
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r)
                    if (lane + 32 * r < g.NP) my_x[lane + 32 * r] = 0.f;
                __syncwarp();
                if (on) my_x[atom] = s;
            }
        }
        cl.sync();
        if (LV) {
            // mean and 1/(8 sigma) of the windows whose left column is this one
            if (lv_left) {
                for (int r0 = lane; r0 + 2 < g.H; r0 += 32) {
                    float v[9];
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        v[d] = my_x[r0 + d];
                        v[3 + d] = x1[r0 + d];
                        v[6 + d] = x2[r0 + d];
                    }
                    float sum = 0.f;
#pragma unroll
                    for (int d = 0; d < 9; ++d) sum += v[d];
                    const float mu = sum * (1.f / 9.f);
                    float ss = 0.f;
#pragma unroll
                    for (int d = 0; d < 9; ++d) ss = fmaf(v[d] - mu, v[d] - mu, ss);
                    const float sigma = sqrtf(fmaf(ss, 0.125f, g.lv_eps2));
                    my_st[r0] = make_float2(mu, sigma > 0.f ? 1.f / (8.f * sigma) : 0.f);
                }
            }
            cl.sync();
        }
        // g = G s - b + c_j lam s - lam (s_left + s_right) at this atom
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        if constexpr (!LV) {
#pragma unroll
            for (int p4 = 0; p4 < KT; p4 += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&mine[p4]);
                acc[0] = fmaf(grow[p4], v.x, acc[0]);
                acc[1] = fmaf(grow[p4 + 1], v.y, acc[1]);
                acc[2] = fmaf(grow[p4 + 2], v.z, acc[2]);
                acc[3] = fmaf(grow[p4 + 3], v.w, acc[3]);
            }
        } else if (live && on) {
#pragma unroll
            for (int p4 = 0; p4 < KT; p4 += 4) {
                const float4 v = *reinterpret_cast<const float4*>(&mine[p4]);
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int p = p4 + e;
                    const float sv = e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w;
                    if (p < sz) acc[e] = fmaf(__ldg(&Gr[p]), sv, acc[e]);
                }
            }
        }
        float nsum = 0.f;
        if (pos_l >= 0) {
            const float* lb = l_remote ? cl.map_shared_rank(&sh_s[par][wpc - 1][0], rank - 1) : sh_s[par][w - 1];
            nsum += lb[pos_l];
        }
        if (pos_r >= 0) {
            const float* rb = r_remote ? cl.map_shared_rank(&sh_s[par][0][0], rank + 1) : sh_s[par][w + 1];
            nsum += rb[pos_r];
        }
        float glv = 0.f;
        if (LV) {
            // pixel gradient of this column, kept in place of its pixels
            // (nobody reads them again before the next step's barrier)
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int i = lane + 32 * r;
                if (i < g.H && in_img) {
                    const float xi = my_x[i];
                    float gi = 0.f;
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        const int r0 = i - d;
                        if (r0 < 0 || r0 + 2 >= g.H) continue;
                        if (lv_self) {
                            const float2 m = my_st[r0];
                            gi = fmaf(xi - m.x, m.y, gi);
                        }
                        if (sm1) {
                            const float2 m = sm1[r0];
                            gi = fmaf(xi - m.x, m.y, gi);
                        }
                        if (sm2) {
                            const float2 m = sm2[r0];
                            gi = fmaf(xi - m.x, m.y, gi);
                        }
                    }
                    my_x[i] = gi;
                }
            }
            __syncwarp();
            // back to the support: (D_S^T gx)_q, a warp sum per atom
            if (g.D) {
                float gxr[NR];
#pragma unroll
                for (int r = 0; r < NR; ++r) gxr[r] = lane + 32 * r < g.H ? my_x[lane + 32 * r] : 0.f;
                int q = 0;
                // four atoms at a time, then four warp sums
                for (; q + 4 <= sz; q += 4) {
                    const float* d0 = g.D + sh_off[w][q];
                    const float* d1 = g.D + sh_off[w][q + 1];
                    const float* d2 = g.D + sh_off[w][q + 2];
                    const float* d3 = g.D + sh_off[w][q + 3];
                    float p0 = 0.f, p1 = 0.f, p2 = 0.f, p3 = 0.f;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = lane + 32 * r;
                        if (i < g.H) {
                            p0 = fmaf(d0[i], gxr[r], p0);
                            p1 = fmaf(d1[i], gxr[r], p1);
                            p2 = fmaf(d2[i], gxr[r], p2);
                            p3 = fmaf(d3[i], gxr[r], p3);
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        p0 += __shfl_xor_sync(0xffffffffu, p0, o);
                        p1 += __shfl_xor_sync(0xffffffffu, p1, o);
                        p2 += __shfl_xor_sync(0xffffffffu, p2, o);
                        p3 += __shfl_xor_sync(0xffffffffu, p3, o);
                    }
                    glv = lane == q ? p0 : lane == q + 1 ? p1 : lane == q + 2 ? p2 : lane == q + 3 ? p3 : glv;
                }
                for (; q < sz; ++q) {
                    const float* dq = g.D + sh_off[w][q];
                    float part = 0.f;
#pragma unroll
                    for (int r = 0; r < NR; ++r) {
                        const int i = lane + 32 * r;
                        if (i < g.H) part = fmaf(dq[i], gxr[r], part);
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
                    if (lane == q) glv = part;
                }
            } else if (on) {
                glv = my_x[atom];
            }
        }
        if (live && on) {
            float gq = ((acc[0] + acc[1]) + (acc[2] + acc[3]) - bb) + fmaf(c_self, s, -g.lam_h * nsum);
            if (LV) gq = fmaf(g.lv_scale, glv, gq);
            const float2 cc = tab[step];
            mo = fmaf(c.beta1, mo, omb1 * gq);
            ve = fmaf(c.beta2, ve, omb2 * gq * gq);
            // sqrt(v) as v * rsqrt(v) (0 stays 0), approximate reciprocal
            const float rt = ve * rsqrtf(fmaxf(ve, 1e-37f));
            s -= cc.x * mo * rcp_approx(fmaf(rt, cc.y, c.eps));
        }
        if (LV) __syncwarp();
    }
    // no CTA leaves while a neighbour may still read its shared memory
    cl.sync();
    if (live) {
        if (on) {
            a.coef[(size_t)b * a.k + lane] = s;
            a.am[(size_t)b * K + lane] = mo;
            a.av[(size_t)b * K + lane] = ve;
        }
        if (lane == 0) {
            a.tau[b] = c.tau0 + c.steps;
            a.n_iter[b] = sz;
        }
    }
}

size_t lv_smem_bytes(int wpc, int NP) { return (size_t)wpc * NP * (sizeof(float) + sizeof(float2)); }

cudaLaunchConfig_t image_config(int W, bool lv, int NP, int images, cudaStream_t s, cudaLaunchAttribute* at) {
    const int csz = ceil_div(W, kImgWarps);
    const int wpc = ceil_div(W, csz);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(images * csz);
    cfg.blockDim = dim3(32 * wpc);
    cfg.dynamicSmemBytes = lv ? lv_smem_bytes(wpc, NP) : 0;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csz;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

template <int KT, bool LV>
cudaError_t prepare_kt(int W, int NP, int* clusters) {
    auto kern = k_clfit_image<KT, LV>;
    cudaError_t e;
    if (ceil_div(W, kImgWarps) > 8 &&
        (e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
        return e;
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = image_config(W, LV, NP, 1, 0, at);
    // the largest size any image needs: the attribute is the kernel's, shared
    // by every plan, so it never shrinks below what another plan launches with
    if (LV && (e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)lv_smem_bytes(kImgWarps, kLvMaxN))) != cudaSuccess)
        return e;
    return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
}

template <bool LV>
cudaError_t prepare_all(int W, int NP, int* least) {
    int n = 0;
    cudaError_t e;
    if ((e = prepare_kt<8, LV>(W, NP, &n)) != cudaSuccess) return e;
    *least = n < *least ? n : *least;
    if ((e = prepare_kt<16, LV>(W, NP, &n)) != cudaSuccess) return e;
    *least = n < *least ? n : *least;
    if ((e = prepare_kt<24, LV>(W, NP, &n)) != cudaSuccess) return e;
    *least = n < *least ? n : *least;
    if ((e = prepare_kt<32, LV>(W, NP, &n)) != cudaSuccess) return e;
    *least = n < *least ? n : *least;
    return cudaSuccess;
}

template <int KT, bool LV>
cudaError_t launch_kt(const IterArgs& a, const ClArgs& c, ImgArgs g, cudaStream_t s) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = image_config(g.W, LV, g.NP, a.B / g.W, s, at);
    g.wpc = (int)cfg.blockDim.x / 32;
    return cudaLaunchKernelEx(&cfg, k_clfit_image<KT, LV>, a, c, g);
}

template <bool LV>
cudaError_t launch_lv(const IterArgs& a, const ClArgs& c, int iter, const ImgArgs& g, cudaStream_t s) {
    // every live column holds iter + 1 atoms during this fit, stopped ones fewer
    switch (round_up(iter + 1, 8)) {
        case 8: return launch_kt<8, LV>(a, c, g, s);
        case 16: return launch_kt<16, LV>(a, c, g, s);
        case 24: return launch_kt<24, LV>(a, c, g, s);
        default: return launch_kt<32, LV>(a, c, g, s);
    }
}

}  // namespace

bool clfit_image_supported(const IterArgs& a, int W, bool lv, int H) {
    return W >= 2 && W <= 16 * kImgWarps && a.B % W == 0 && a.k <= 32 && (!lv || (H >= 1 && H <= kLvMaxN));
}

// Allows the cluster size (and, with LV, the shared memory) the image needs
// and checks that such clusters fit on this device (*ok = 0: they do not).
// Call outside stream capture, before the first launch for this shape.
cudaError_t clfit_image_prepare(int W, bool lv, int H, int* ok) {
    *ok = 0;
    int least = 1 << 30;
    const cudaError_t e = lv ? prepare_all<true>(W, round_up(H, 32), &least)
                             : prepare_all<false>(W, 0, &least);
    if (e != cudaSuccess) return e;
    *ok = least >= 1;
    return cudaSuccess;
}

cudaError_t launch_clfit_image(const IterArgs& a, const ClArgs& c, int iter, int W, float lam_h, float lv_scale,
                               float lv_eps, const float* D, int H, int ldd, cudaStream_t s) {
    ImgArgs g;
    g.W = W;
    g.wpc = 0;
    g.lam_h = lam_h;
    g.lv_scale = lv_scale;
    g.lv_eps2 = lv_eps * lv_eps;
    g.D = D;
    g.H = H;
    g.ldd = ldd;
    g.NP = round_up(H, 32);
    return lv_scale != 0.f ? launch_lv<true>(a, c, iter, g, s) : launch_lv<false>(a, c, iter, g, s);
}

}  // namespace cs
