// Learned block preconditioner: a 3-layer perceptron (bfloat16 weights,
// float32 accumulation) that maps features of each QN block of the local
// problem to two coefficients (gamma, delta) of the block's initial guess
//   x0_B = gamma_B * x_warm,B + delta_B * (D^-1 b)_B
// (x_warm: the current two-site tensor, D: the Jacobi diagonal, b = -g).
// The plain Jacobi-PCG stays the solver and the fallback: the learned guess
// is used only when its float64 residual is smaller than the warm start's,
// and CG then converges to the same tolerance, so the energy is unchanged.
#pragma once
#include <vector>

#include "core.h"
#include "kernels.h"

namespace mpspt {

struct Mlp {
    int nin = 0, width = 0, nout = 0;
    cudaStream_t st = 0;
    DBuf W[3], b[3], Wb[3], mW[3], vW[3], mb[3], vb[3], gW[3], gb[3];
    DBuf X, H1, H2, Y, T, dY, dH2, dH1, rowloss;
    int cap = 0, step = 0;

    Mlp(int nin_, int width_, int nout_, unsigned long long seed, cudaStream_t st_);
    int in_of(int l) const { return l == 0 ? nin : width; }
    int out_of(int l) const { return l == 2 ? nout : width; }
    size_t wn(int l) const { return (size_t)in_of(l) * out_of(l); }
    void set_params(const float* const* Wh, const float* const* bh);
    void get_params(float* const* Wh, float* const* bh) const;
    void ensure(int B);
    void forward(int B, const float* Xd, float* Yd);          // device in/out
    float gradient(int B, const float* Xd, const float* Td);  // fills gW, gb; returns loss
    void adam(float lr);
    float train(int n, const float* Xh, const float* Th, int epochs, int batch, float lr);
};

}  // namespace mpspt
