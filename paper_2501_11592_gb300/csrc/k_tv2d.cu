// CLOMP fit with the total-variation prior of an image (Eq. 6).  The batch is
// a sequence of images of W consecutive columns, column j of an image being
// the signal x_j = D s_j.  The prior's vertical part is the 1-D form of
// Eq. 5 per column and already sits in A^T A (k_prior.cu), so it reaches the
// per-signal Gram matrices G = A_S^T A_S + (2w/H)(Delta D_S)^T(Delta D_S).
// Its horizontal part, (w/W) sum_j ||x_j - x_{j+1}||^2, couples neighbouring
// columns; for a basis with orthonormal columns (D^T D = I: the DCT, or no
// basis) it equals (w/W) sum_j ||s_j - s_{j+1}||^2, whose gradient with
// respect to column j's support coefficients is
//   (2w/W) (c_j s_j - s_{j-1}|_{S_j} - s_{j+1}|_{S_j}),
// c_j the number of neighbours (1 at the image's edges, else 2) and
// s_{j+-1}|_{S_j} the neighbour's coefficients at the atoms of S_j (zero where
// the neighbour has not selected the atom).
//
// The columns of an image take their Adam steps together, each step's
// gradients from the coefficients before it, so an image is one thread-block
// cluster: one warp per column, lane q owning coordinate q (row q of G in
// registers), the columns' coefficient vectors published in shared memory
// every step (double-buffered) and read across the cluster through
// distributed shared memory at the CTA boundaries.  One cluster barrier per
// step orders publication and reads.  Stopped columns keep their
// coefficients and still serve as neighbours.
#include <cooperative_groups.h>

#include "k_fit.cuh"

namespace cg = cooperative_groups;

namespace cs {
namespace {

constexpr int kTvWarps = 32;   // columns (warps) per CTA at most

template <int KT>
__global__ void __launch_bounds__(1024, 1)
    k_clfit_tv2d(IterArgs a, ClArgs c, int W, int wpc, float lam_h) {
    static_assert(KT % 8 == 0 && KT >= 8 && KT <= 32, "one coordinate per lane");
    cg::cluster_group cl = cg::this_cluster();
    __shared__ __align__(16) float sh_s[2][kTvWarps][KT];
    __shared__ float2 sh_tab[kAdamStaged];
    const float2* tab = stage_adam(c, sh_tab);
    __syncthreads();

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int rank = (int)cl.block_rank(), csz = (int)cl.num_blocks();
    const int img = blockIdx.x / csz;
    const int col = rank * wpc + w;                 // column within the image
    const bool in_img = col < W;
    const int b = img * W + (in_img ? col : 0);
    const int K = a.kmax;
    const bool live = in_img && a.status[b] < 0;
    // support size: a live column got this iteration's atom from the selection
    const int sz = in_img ? a.n_iter[b] + (live ? 1 : 0) : 0;
    const bool on = lane < sz;

    float grow[KT];
    {
        const float* Gr = a.G + ((size_t)b * K + (on ? lane : 0)) * K;
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
    if (live && on) {
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
    const float c_self = lam_h * (float)((col > 0 ? 1 : 0) + (col < W - 1 ? 1 : 0));
    // neighbours' buffers: the next warp of this CTA, or the edge warp of the
    // neighbouring CTA of the cluster
    const bool l_remote = w == 0, r_remote = w == wpc - 1;
    const float omb1 = 1.f - c.beta1, omb2 = 1.f - c.beta2;

    for (int step = 0; step < c.steps; ++step) {
        const int par = step & 1;
        float* mine = sh_s[par][w];
        if (lane < KT) mine[lane] = s;
        cl.sync();
        // g = G s - b + c_j lam s - lam (s_left + s_right) at this atom
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int p4 = 0; p4 < KT; p4 += 4) {
            const float4 v = *reinterpret_cast<const float4*>(&mine[p4]);
            acc[0] = fmaf(grow[p4], v.x, acc[0]);
            acc[1] = fmaf(grow[p4 + 1], v.y, acc[1]);
            acc[2] = fmaf(grow[p4 + 2], v.z, acc[2]);
            acc[3] = fmaf(grow[p4 + 3], v.w, acc[3]);
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
        if (live && on) {
            const float gq = ((acc[0] + acc[1]) + (acc[2] + acc[3]) - bb) + fmaf(c_self, s, -lam_h * nsum);
            const float2 cc = tab[step];
            mo = fmaf(c.beta1, mo, omb1 * gq);
            ve = fmaf(c.beta2, ve, omb2 * gq * gq);
            // sqrt(v) as v * rsqrt(v) (0 stays 0), approximate reciprocal
            const float rt = ve * rsqrtf(fmaxf(ve, 1e-37f));
            s -= cc.x * mo * rcp_approx(fmaf(rt, cc.y, c.eps));
        }
    }
    // no CTA leaves while a neighbour may still read its buffers
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

cudaLaunchConfig_t tv2d_config(int W, int images, cudaStream_t s, cudaLaunchAttribute* at) {
    const int csz = ceil_div(W, kTvWarps);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(images * csz);
    cfg.blockDim = dim3(32 * ceil_div(W, csz));
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = csz;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cfg;
}

template <int KT>
cudaError_t prepare_kt(int W, int* clusters) {
    auto kern = k_clfit_tv2d<KT>;
    if (ceil_div(W, kTvWarps) > 8) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = tv2d_config(W, 1, 0, at);
    return cudaOccupancyMaxActiveClusters(clusters, kern, &cfg);
}

template <int KT>
cudaError_t launch_kt(const IterArgs& a, const ClArgs& c, int W, float lam_h, cudaStream_t s) {
    cudaLaunchAttribute at[1];
    const cudaLaunchConfig_t cfg = tv2d_config(W, a.B / W, s, at);
    const int wpc = (int)cfg.blockDim.x / 32;
    return cudaLaunchKernelEx(&cfg, k_clfit_tv2d<KT>, a, c, W, wpc, lam_h);
}

}  // namespace

bool clfit_tv2d_supported(const IterArgs& a, int W) {
    return W >= 2 && W <= 16 * kTvWarps && a.B % W == 0 && a.k <= 32;
}

// Allows the cluster size the image width needs and checks that such
// clusters fit on this device (*ok = 0: they do not).  Call outside stream
// capture, before the first launch for this width.
cudaError_t clfit_tv2d_prepare(int W, int* ok) {
    *ok = 0;
    int least = 1 << 30;
    int n = 0;
    cudaError_t e;
    if ((e = prepare_kt<8>(W, &n)) != cudaSuccess) return e;
    least = n < least ? n : least;
    if ((e = prepare_kt<16>(W, &n)) != cudaSuccess) return e;
    least = n < least ? n : least;
    if ((e = prepare_kt<24>(W, &n)) != cudaSuccess) return e;
    least = n < least ? n : least;
    if ((e = prepare_kt<32>(W, &n)) != cudaSuccess) return e;
    least = n < least ? n : least;
    *ok = least >= 1;
    return cudaSuccess;
}

cudaError_t launch_clfit_tv2d(const IterArgs& a, const ClArgs& c, int iter, int W, float lam_h, cudaStream_t s) {
    // every live column holds iter + 1 atoms during this fit, stopped ones fewer
    switch (round_up(iter + 1, 8)) {
        case 8: return launch_kt<8>(a, c, W, lam_h, s);
        case 16: return launch_kt<16>(a, c, W, lam_h, s);
        case 24: return launch_kt<24>(a, c, W, lam_h, s);
        default: return launch_kt<32>(a, c, W, lam_h, s);
    }
}

}  // namespace cs
