// Learned block preconditioner: network training and inference on the GPU.
#include "learned.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <random>

namespace mpspt {

Mlp::Mlp(int nin_, int width_, int nout_, unsigned long long seed, cudaStream_t st_)
    : nin(nin_), width(width_), nout(nout_), st(st_) {
    require(nin >= 1 && width >= 1 && nout >= 1, "invalid network shape");
    std::mt19937_64 gen(seed);
    for (int l = 0; l < 3; ++l) {
        const size_t n = wn(l);
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (float)in_of(l)));
        std::vector<float> w(n);
        for (auto& v : w) v = nd(gen);
        std::vector<float> z(out_of(l), 0.f), zn(n, 0.f);
        upload(W[l], w, st);
        upload(b[l], z, st);
        upload(mW[l], zn, st);
        upload(vW[l], zn, st);
        upload(mb[l], z, st);
        upload(vb[l], z, st);
        gW[l].ensure(n * sizeof(float) + 16, st);
        gb[l].ensure(out_of(l) * sizeof(float) + 16, st);
        Wb[l].ensure(n * 2 + 16, st);
        mlp_to_bf16((int)n, W[l].as<float>(), Wb[l].get(), st);
    }
    MPSPT_CUDA(cudaStreamSynchronize(st));
}

void Mlp::set_params(const float* const* Wh, const float* const* bh) {
    for (int l = 0; l < 3; ++l) {
        MPSPT_CUDA(cudaMemcpyAsync(W[l].get(), Wh[l], wn(l) * sizeof(float), cudaMemcpyHostToDevice, st));
        MPSPT_CUDA(cudaMemcpyAsync(b[l].get(), bh[l], out_of(l) * sizeof(float), cudaMemcpyHostToDevice, st));
        mlp_to_bf16((int)wn(l), W[l].as<float>(), Wb[l].get(), st);
        MPSPT_CUDA(cudaMemsetAsync(mW[l].get(), 0, wn(l) * sizeof(float), st));
        MPSPT_CUDA(cudaMemsetAsync(vW[l].get(), 0, wn(l) * sizeof(float), st));
        MPSPT_CUDA(cudaMemsetAsync(mb[l].get(), 0, out_of(l) * sizeof(float), st));
        MPSPT_CUDA(cudaMemsetAsync(vb[l].get(), 0, out_of(l) * sizeof(float), st));
    }
    step = 0;
    MPSPT_CUDA(cudaStreamSynchronize(st));
}

void Mlp::get_params(float* const* Wh, float* const* bh) const {
    for (int l = 0; l < 3; ++l) {
        MPSPT_CUDA(cudaMemcpyAsync(Wh[l], W[l].get(), wn(l) * sizeof(float), cudaMemcpyDeviceToHost, st));
        MPSPT_CUDA(cudaMemcpyAsync(bh[l], b[l].get(), out_of(l) * sizeof(float), cudaMemcpyDeviceToHost, st));
    }
    MPSPT_CUDA(cudaStreamSynchronize(st));
}

void Mlp::ensure(int B) {
    if (B <= cap) return;
    cap = B;
    const size_t f = sizeof(float);
    X.ensure((size_t)B * nin * f + 16, st);
    T.ensure((size_t)B * nout * f + 16, st);
    Y.ensure((size_t)B * nout * f + 16, st);
    dY.ensure((size_t)B * nout * f + 16, st);
    H1.ensure((size_t)B * width * f + 16, st);
    H2.ensure((size_t)B * width * f + 16, st);
    dH1.ensure((size_t)B * width * f + 16, st);
    dH2.ensure((size_t)B * width * f + 16, st);
    rowloss.ensure((size_t)B * f + 16, st);
}

void Mlp::forward(int B, const float* Xd, float* Yd) {
    ensure(B);
    // H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3
    mlp_gemm_bf16w(B, width, nin, Xd, nin, false, Wb[0].get(), nin, true, H1.as<float>(), width, b[0].as<float>(),
                   nullptr, 2, st);
    mlp_gemm_bf16w(B, width, width, H1.as<float>(), width, false, Wb[1].get(), width, true, H2.as<float>(), width,
                   b[1].as<float>(), nullptr, 2, st);
    mlp_gemm_bf16w(B, nout, width, H2.as<float>(), width, false, Wb[2].get(), width, true, Yd, nout,
                   b[2].as<float>(), nullptr, 1, st);
}

float Mlp::gradient(int B, const float* Xd, const float* Td) {
    ensure(B);
    forward(B, Xd, Y.as<float>());
    mlp_mse(B, nout, Y.as<float>(), Td, dY.as<float>(), rowloss.as<float>(), st);
    // layer 3
    mlp_gemm(nout, width, B, dY.as<float>(), nout, true, H2.as<float>(), width, false, gW[2].as<float>(), width,
             nullptr, nullptr, 0, st);
    mlp_colsum(B, nout, dY.as<float>(), gb[2].as<float>(), st);
    mlp_gemm_bf16w(B, width, nout, dY.as<float>(), nout, false, Wb[2].get(), width, false, dH2.as<float>(), width,
                   nullptr, H2.as<float>(), 3, st);
    // layer 2
    mlp_gemm(width, width, B, dH2.as<float>(), width, true, H1.as<float>(), width, false, gW[1].as<float>(), width,
             nullptr, nullptr, 0, st);
    mlp_colsum(B, width, dH2.as<float>(), gb[1].as<float>(), st);
    mlp_gemm_bf16w(B, width, width, dH2.as<float>(), width, false, Wb[1].get(), width, false, dH1.as<float>(),
                   width, nullptr, H1.as<float>(), 3, st);
    // layer 1
    mlp_gemm(width, nin, B, dH1.as<float>(), width, true, Xd, nin, false, gW[0].as<float>(), nin, nullptr, nullptr,
             0, st);
    mlp_colsum(B, width, dH1.as<float>(), gb[0].as<float>(), st);
    std::vector<float> rl(B);
    MPSPT_CUDA(cudaMemcpyAsync(rl.data(), rowloss.get(), (size_t)B * sizeof(float), cudaMemcpyDeviceToHost, st));
    MPSPT_CUDA(cudaStreamSynchronize(st));
    double s = 0.0;
    for (float v : rl) s += v;
    return (float)s;
}

void Mlp::adam(float lr) {
    ++step;
    for (int l = 0; l < 3; ++l) {
        mlp_adam((int)wn(l), W[l].as<float>(), gW[l].as<float>(), mW[l].as<float>(), vW[l].as<float>(), Wb[l].get(),
                 lr, step, st);
        mlp_adam(out_of(l), b[l].as<float>(), gb[l].as<float>(), mb[l].as<float>(), vb[l].as<float>(), nullptr, lr,
                 step, st);
    }
}

float Mlp::train(int n, const float* Xh, const float* Th, int epochs, int batch, float lr) {
    require(n >= 1 && epochs >= 1 && batch >= 1, "invalid training arguments");
    batch = std::min(batch, n);
    DBuf Xall, Tall;
    std::vector<float> xs(Xh, Xh + (size_t)n * nin), ts(Th, Th + (size_t)n * nout);
    upload(Xall, xs, st);
    upload(Tall, ts, st);
    float last = 0.f;
    for (int e = 0; e < epochs; ++e) {
        double tot = 0.0;
        int nb = 0;
        for (int o = 0; o + batch <= n; o += batch) {
            tot += gradient(batch, Xall.as<float>() + (size_t)o * nin, Tall.as<float>() + (size_t)o * nout);
            adam(lr);
            ++nb;
        }
        last = (float)(tot / std::max(1, nb));
    }
    MPSPT_CUDA(cudaStreamSynchronize(st));
    return last;
}

}  // namespace mpspt
