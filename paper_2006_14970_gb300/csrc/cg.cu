// Converged reference: the minimiser of the global cost whose per-pixel minimisation the
// method iterates (the local cost of Section III-C summed over the pixels, each
// 4-neighbour edge once), by preconditioned conjugate gradients in float64. Per channel,
// grad E = 0 is H x = b with x = (F, B), b = (alpha I, (1 - alpha) I) and
//   (H x)_F,i = alpha_i (alpha_i F_i + (1 - alpha_i) B_i) + sum_j d_ij (F_i - F_j)
//   (H x)_B,i = (1 - alpha_i) (alpha_i F_i + (1 - alpha_i) B_i) + sum_j d_ij (B_i - B_j)
// over the in-image neighbours j, d_ij = eps_r + omega |alpha_i - alpha_j|. The three
// channels form one block-diagonal system (one CG, inner products over all channels).
// The preconditioner inverts each pixel's 2 x 2 diagonal block of H (block Jacobi: the
// same 2 x 2 solve as the method's update, without the clamp).
//
// One thread per pixel, all channels. Every inner product is a per-block partial followed
// by a one-block kernel that adds the partials in a fixed order and forms the CG scalars
// on the device, so an iteration is four launches and needs no host round trip.
#include "fgml_internal.h"

namespace fgml {
namespace {

constexpr int kThreads = 256;

struct Pix {
    int i;            // pixel index
    double a;         // alpha_i
    int nb[4];        // neighbour pixel indices (valid where on[k])
    bool on[4];
    double d[4];      // edge weights
    double S;         // sum of the weights
};

template <typename T>
__device__ __forceinline__ double alpha_at(const CgArgs &g, int x, int y) {
    return (double)ld_elem(static_cast<const T *>(g.A) + (long long)y * g.A_pitch + x);
}

template <typename T>
__device__ __forceinline__ Pix pixel(const CgArgs &g, int i) {
    Pix p;
    const int x = i % g.w, y = i / g.w;
    p.i = i;
    p.a = alpha_at<T>(g, x, y);
    const int xs[4] = {x - 1, x + 1, x, x}, ys[4] = {y, y, y - 1, y + 1};
    p.S = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p.on[k] = xs[k] >= 0 && xs[k] < g.w && ys[k] >= 0 && ys[k] < g.h;
        p.nb[k] = p.on[k] ? ys[k] * g.w + xs[k] : i;
        p.d[k] = p.on[k] ? g.eps + g.omega * fabs(p.a - alpha_at<T>(g, xs[k], ys[k])) : 0.0;
        p.S += p.d[k];
    }
    return p;
}

// (H v)_i for channel c, with v read through vf(j) (F part) and vb(j) (B part).
template <typename VF, typename VB>
__device__ __forceinline__ void apply_h(const Pix &p, VF vf, VB vb, double &hf, double &hb) {
    const double fi = vf(p.i), bi = vb(p.i);
    const double comp = p.a * fi + (1.0 - p.a) * bi;
    double lf = 0.0, lb = 0.0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (!p.on[k]) continue;
        lf += p.d[k] * (fi - vf(p.nb[k]));
        lb += p.d[k] * (bi - vb(p.nb[k]));
    }
    hf = p.a * comp + lf;
    hb = (1.0 - p.a) * comp + lb;
}

// z = D_i^-1 r for the pixel's 2 x 2 diagonal block D_i (a tiny multiple of the identity
// keeps it invertible where it is singular; the preconditioner does not change the
// solution)
__device__ __forceinline__ void precond(const Pix &p, double rf, double rb, double &zf, double &zb) {
    const double be = 1.0 - p.a;
    const double d00 = p.a * p.a + p.S + 1e-12, d11 = be * be + p.S + 1e-12, d01 = p.a * be;
    const double inv = 1.0 / (d00 * d11 - d01 * d01);
    zf = (d11 * rf - d01 * rb) * inv;
    zb = (d00 * rb - d01 * rf) * inv;
}

template <typename T>
__device__ __forceinline__ double image_at(const CgArgs &g, int i, int c) {
    const int x = i % g.w, y = i / g.w;
    return (double)ld_elem(static_cast<const T *>(g.I) + (long long)y * g.I_pitch + 3 * x + c);
}

__device__ __forceinline__ void store_partials(const CgArgs &g, double v0, double v1, double v2,
                                               double *red) {
    v0 = block_sum_d(v0, red);
    if (threadIdx.x == 0) g.partials[3 * blockIdx.x + 0] = v0;
    v1 = block_sum_d(v1, red);
    if (threadIdx.x == 0) g.partials[3 * blockIdx.x + 1] = v1;
    v2 = block_sum_d(v2, red);
    if (threadIdx.x == 0) g.partials[3 * blockIdx.x + 2] = v2;
}

// r = b - H x, z = M^-1 r, p = z; partials (r.z, b.b, r.r)
template <typename T>
__global__ void __launch_bounds__(kThreads) cg_start_kernel(const CgArgs g, double *pv) {
    __shared__ double red[kThreads / 32];
    const long long n = (long long)g.w * g.h;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double rz = 0.0, bb = 0.0, rr = 0.0;
    if (i < n) {
        const Pix p = pixel<T>(g, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            double hf, hb;
            apply_h(p, [&](int j) { return g.x[3 * j + c]; },
                    [&](int j) { return g.x[3 * n + 3 * j + c]; }, hf, hb);
            const double Ii = image_at<T>(g, i, c);
            const double bf = p.a * Ii, bbv = (1.0 - p.a) * Ii;
            const double rf = bf - hf, rb = bbv - hb;
            double zf, zb;
            precond(p, rf, rb, zf, zb);
            g.r[3 * i + c] = rf;
            g.r[3 * n + 3 * i + c] = rb;
            g.z[3 * i + c] = zf;
            g.z[3 * n + 3 * i + c] = zb;
            pv[3 * i + c] = zf;
            pv[3 * n + 3 * i + c] = zb;
            rz += rf * zf + rb * zb;
            bb += bf * bf + bbv * bbv;
            rr += rf * rf + rb * rb;
        }
    }
    store_partials(g, rz, bb, rr, red);
}

// p_new = z + beta p_old (also at the neighbours, from p_old), q = H p_new; partial p.q
template <typename T>
__global__ void __launch_bounds__(kThreads) cg_apply_kernel(const CgArgs g, const double *p_old,
                                                            double *p_new) {
    __shared__ double red[kThreads / 32];
    const long long n = (long long)g.w * g.h;
    const double beta = g.sc->beta;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double pq = 0.0;
    if (i < n) {
        const Pix p = pixel<T>(g, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            auto pf = [&](int j) { return g.z[3 * j + c] + beta * p_old[3 * j + c]; };
            auto pb = [&](int j) { return g.z[3 * n + 3 * j + c] + beta * p_old[3 * n + 3 * j + c]; };
            double hf, hb;
            apply_h(p, pf, pb, hf, hb);
            const double vf = pf(i), vb = pb(i);
            p_new[3 * i + c] = vf;
            p_new[3 * n + 3 * i + c] = vb;
            g.q[3 * i + c] = hf;
            g.q[3 * n + 3 * i + c] = hb;
            pq += vf * hf + vb * hb;
        }
    }
    store_partials(g, pq, 0.0, 0.0, red);
}

// x += alpha p, r -= alpha q, z = M^-1 r; partials (r.z, -, r.r)
template <typename T>
__global__ void __launch_bounds__(kThreads) cg_update_kernel(const CgArgs g, const double *pv) {
    __shared__ double red[kThreads / 32];
    const long long n = (long long)g.w * g.h;
    const double al = g.sc->alpha;
    const int i = blockIdx.x * kThreads + threadIdx.x;
    double rz = 0.0, rr = 0.0;
    if (i < n) {
        const Pix p = pixel<T>(g, i);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long jf = 3 * i + c, jb = 3 * n + 3 * i + c;
            g.x[jf] += al * pv[jf];
            g.x[jb] += al * pv[jb];
            const double rf = g.r[jf] - al * g.q[jf], rb = g.r[jb] - al * g.q[jb];
            g.r[jf] = rf;
            g.r[jb] = rb;
            double zf, zb;
            precond(p, rf, rb, zf, zb);
            g.z[jf] = zf;
            g.z[jb] = zb;
            rz += rf * zf + rb * zb;
            rr += rf * rf + rb * rb;
        }
    }
    store_partials(g, rz, 0.0, rr, red);
}

// The sums of the partials, then the CG scalars. mode 0: after cg_start; 1: after
// cg_apply (alpha); 2: after cg_update (beta); 3: after the true-residual pass.
__global__ void __launch_bounds__(kThreads) cg_reduce_kernel(const double *partials, int nb,
                                                             CgScalars *sc, int mode) {
    __shared__ double red[kThreads / 32];
    double v[3];
    for (int k = 0; k < 3; ++k) {
        double t = 0.0;
        for (int b = threadIdx.x; b < nb; b += kThreads) t += partials[3 * b + k];
        v[k] = block_sum_d(t, red);
    }
    if (threadIdx.x != 0) return;
    if (mode == 0) {
        sc->rz = v[0];
        sc->bb = v[1];
        sc->rr = v[2];
        sc->beta = 0.0;
    } else if (mode == 1) {
        sc->pq = v[0];
        sc->alpha = v[0] > 0.0 ? sc->rz / v[0] : 0.0;
    } else if (mode == 2) {
        sc->beta = sc->rz > 0.0 ? v[0] / sc->rz : 0.0;
        sc->rz = v[0];
        sc->rr = v[2];
    } else {
        sc->rr = v[2];
    }
}

template <typename T>
cudaError_t start_t(const CgArgs &a, double *p, cudaStream_t s) {
    const int nb = cg_blocks(a.w, a.h);
    cg_start_kernel<T><<<nb, kThreads, 0, s>>>(a, p);
    cg_reduce_kernel<<<1, kThreads, 0, s>>>(a.partials, nb, a.sc, 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t iterate_t(const CgArgs &a, const double *p_old, double *p_new, cudaStream_t s) {
    const int nb = cg_blocks(a.w, a.h);
    cg_apply_kernel<T><<<nb, kThreads, 0, s>>>(a, p_old, p_new);
    cg_reduce_kernel<<<1, kThreads, 0, s>>>(a.partials, nb, a.sc, 1);
    cg_update_kernel<T><<<nb, kThreads, 0, s>>>(a, p_new);
    cg_reduce_kernel<<<1, kThreads, 0, s>>>(a.partials, nb, a.sc, 2);
    return cudaGetLastError();
}

template <typename T>
cudaError_t residual_t(const CgArgs &a, cudaStream_t s) {
    const int nb = cg_blocks(a.w, a.h);
    cg_start_kernel<T><<<nb, kThreads, 0, s>>>(a, a.q);   // q as scratch for p
    cg_reduce_kernel<<<1, kThreads, 0, s>>>(a.partials, nb, a.sc, 3);
    return cudaGetLastError();
}

}  // namespace

int cg_blocks(int w, int h) { return (int)(((long long)w * h + kThreads - 1) / kThreads); }

cudaError_t cg_start(int dtype, const CgArgs &a, double *p, cudaStream_t s) {
    switch (dtype) {
        case kF32: return start_t<float>(a, p, s);
        case kBF16: return start_t<__nv_bfloat16>(a, p, s);
        case kF16: return start_t<__half>(a, p, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t cg_iterate(int dtype, const CgArgs &a, const double *p_old, double *p_new,
                       cudaStream_t s) {
    switch (dtype) {
        case kF32: return iterate_t<float>(a, p_old, p_new, s);
        case kBF16: return iterate_t<__nv_bfloat16>(a, p_old, p_new, s);
        case kF16: return iterate_t<__half>(a, p_old, p_new, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t cg_true_residual(int dtype, const CgArgs &a, cudaStream_t s) {
    switch (dtype) {
        case kF32: return residual_t<float>(a, s);
        case kBF16: return residual_t<__nv_bfloat16>(a, s);
        case kF16: return residual_t<__half>(a, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace fgml
