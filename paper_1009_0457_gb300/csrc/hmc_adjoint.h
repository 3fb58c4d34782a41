// Arguments and launchers of the adjoint kernels (k_adjoint.cu); single replica.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hmc {

template <typename T>
struct AdjArgs {
    const uint4 *spins;   // block layout
    const T *ctab;        // C'(q), 21 entries padded to 24
    const T *rtab;        // rotated basis tensors R_1, R_2, R_3 per orientation, 3 x 24
    const T *wtab;        // Voigt weights of the three crystal axes a_m (a_m.x.a_m = w_m.x), 20 per orientation
    double *partials;     // per-CTA partial sums
    T ebar[6];            // mean strain of the forward state
    int nx, ny, nz, nbx, nby, nbz, nblk;
};

template <typename T>
cudaError_t launch_adj_params(const AdjArgs<T> &a, const T *lam, const T *u, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_terminal(const AdjArgs<T> &a, const T *u, const T *g, T gW, T *w, T *fcell, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_gather(const AdjArgs<T> &a, const T *fcell, T scale, T *out, cudaStream_t s);
template <typename T>
cudaError_t launch_adj_lambda(long long n, const T *x, T damping, T *lam, cudaStream_t s);
cudaError_t launch_adj_reduce(const double *partials, int nparts, int nv, int stride, double scale, double *out,
                              cudaStream_t s);

}  // namespace hmc
