// CPU ORACLE -- TEST INFRASTRUCTURE ONLY (see oracle_internal.h).
//
// The learned proposal (a project addition, not in the paper): a small MLP
// maps a bin's position and normal to a distribution over the N x N = 32 x 32
// cells of the concentric octahedral grid, trained to match the SVO-traced
// field of Alg. 3 with the KL divergence KL(q || softmax(z)).
//
// Features (78): p^ = (p - lo) / S in [0, 1]^3; for k = 0..11: sin(2^k pi p^)
// and cos(2^k pi p^) (3 + 3 each); the normal n (3).  Network: 78 -> 64 -> 64
// -> 64 -> 1024, ReLU on the hidden layers, softmax over the 1024 logits.
//
// Parameters, flat float32 in this order: W1[64][80] (inputs padded to 80 with
// zero columns), b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[1024][64],
// b4[1024].  Arithmetic in binary64; with `bf16` set, every stored weight,
// input feature, hidden activation and logit gradient is rounded to bfloat16
// (round to nearest even) at the points where the kernels store bfloat16.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace orc {

constexpr int kIn = 80, kFeat = 78, kHid = 64, kOut = 1024;
constexpr size_t kOffW1 = 0, kOffB1 = kOffW1 + kHid * kIn, kOffW2 = kOffB1 + kHid, kOffB2 = kOffW2 + kHid * kHid,
                 kOffW3 = kOffB2 + kHid, kOffB3 = kOffW3 + kHid * kHid, kOffW4 = kOffB3 + kHid,
                 kOffB4 = kOffW4 + (size_t)kOut * kHid, kParams = kOffB4 + kOut;

// round a binary32 value to the nearest bfloat16 (ties to even), as a float
static float bf16_round(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return f;  // inf / nan unchanged
    u += 0x7fffu + ((u >> 16) & 1u);
    u &= 0xffff0000u;
    float r;
    std::memcpy(&r, &u, 4);
    return r;
}
static double rnd(double x, bool bf16) { return bf16 ? (double)bf16_round((float)x) : x; }

void mlp_features(const float* pos, const float* nrm, const float lo[3], float S, double* out) {
    double ph[3];
    for (int a = 0; a < 3; ++a) ph[a] = ((double)pos[a] - (double)lo[a]) / (double)S;
    int j = 0;
    for (int a = 0; a < 3; ++a) out[j++] = ph[a];
    for (int k = 0; k < 12; ++k) {
        const double f = std::ldexp(1.0, k);
        for (int a = 0; a < 3; ++a) out[j++] = std::sin(M_PI * std::fmod(f * ph[a], 2.0));
        for (int a = 0; a < 3; ++a) out[j++] = std::cos(M_PI * std::fmod(f * ph[a], 2.0));
    }
    for (int a = 0; a < 3; ++a) out[j++] = nrm[a];
    out[j++] = 0.0;
    out[j++] = 0.0;
}

struct Fwd {
    std::vector<double> x, h1, h2, h3, z, p;
};

static void dense(const std::vector<double>& W, const double* b, const double* in, int nin, int nout, double* out) {
    for (int o = 0; o < nout; ++o) {
        double s = 0.0;
        for (int i = 0; i < nin; ++i) s += W[(size_t)o * nin + i] * in[i];
        out[o] = s + b[o];
    }
}

static void forward_one(const std::vector<double>* W, const double* const* b, const float* pos, const float* nrm,
                        const float lo[3], float S, bool bf16, Fwd& f) {
    f.x.assign(kIn, 0.0);
    mlp_features(pos, nrm, lo, S, f.x.data());
    for (int i = 0; i < kIn; ++i) f.x[i] = rnd(f.x[i], bf16);
    f.h1.assign(kHid, 0.0);
    f.h2.assign(kHid, 0.0);
    f.h3.assign(kHid, 0.0);
    f.z.assign(kOut, 0.0);
    f.p.assign(kOut, 0.0);
    dense(W[0], b[0], f.x.data(), kIn, kHid, f.h1.data());
    for (double& v : f.h1) v = rnd(v > 0 ? v : 0.0, bf16);
    dense(W[1], b[1], f.h1.data(), kHid, kHid, f.h2.data());
    for (double& v : f.h2) v = rnd(v > 0 ? v : 0.0, bf16);
    dense(W[2], b[2], f.h2.data(), kHid, kHid, f.h3.data());
    for (double& v : f.h3) v = rnd(v > 0 ? v : 0.0, bf16);
    dense(W[3], b[3], f.h3.data(), kHid, kOut, f.z.data());
    double m = f.z[0];
    for (double v : f.z) m = v > m ? v : m;
    double s = 0.0;
    for (int c = 0; c < kOut; ++c) s += (f.p[c] = std::exp(f.z[c] - m));
    for (double& v : f.p) v /= s;
}

static void unpack(const float* params, bool bf16, std::vector<double>* W, std::vector<double>* B) {
    const size_t offW[4] = {kOffW1, kOffW2, kOffW3, kOffW4}, offB[4] = {kOffB1, kOffB2, kOffB3, kOffB4};
    const size_t nW[4] = {(size_t)kHid * kIn, (size_t)kHid * kHid, (size_t)kHid * kHid, (size_t)kOut * kHid};
    const size_t nB[4] = {kHid, kHid, kHid, kOut};
    for (int l = 0; l < 4; ++l) {
        W[l].resize(nW[l]);
        B[l].resize(nB[l]);
        for (size_t i = 0; i < nW[l]; ++i) W[l][i] = rnd(params[offW[l] + i], bf16);
        for (size_t i = 0; i < nB[l]; ++i) B[l][i] = params[offB[l] + i];
    }
}

}  // namespace orc

using namespace orc;

extern "C" {

size_t orc_mlp_num_params(void) { return kParams; }

// the bfloat16 rounding used by the emulation, element by element
void orc_bf16_round(const float* x, size_t n, float* out) {
    for (size_t i = 0; i < n; ++i) out[i] = bf16_round(x[i]);
}

void orc_mlp_features(const float* pos, const float* nrm, size_t n, const float* lo, float S, double* out) {
    for (size_t i = 0; i < n; ++i) mlp_features(pos + 3 * i, nrm + 3 * i, lo, S, out + kIn * i);
}

// logits and probabilities of n samples
void orc_mlp_forward(const float* params, const float* pos, const float* nrm, size_t n, const float* lo, float S,
                     int bf16, double* logits, double* probs) {
    std::vector<double> W[4], B[4];
    unpack(params, bf16 != 0, W, B);
    const double* b[4] = {B[0].data(), B[1].data(), B[2].data(), B[3].data()};
    Fwd f;
    for (size_t i = 0; i < n; ++i) {
        forward_one(W, b, pos + 3 * i, nrm + 3 * i, lo, S, bf16 != 0, f);
        if (logits) std::memcpy(logits + kOut * i, f.z.data(), kOut * 8);
        if (probs) std::memcpy(probs + kOut * i, f.p.data(), kOut * 8);
    }
}

}  // extern "C"

namespace orc {

// The per-sample intermediates of orc_mlp_grad, each [n][width] in binary64
// (bf16-rounded where the kernels store bfloat16); any pointer may be NULL.
struct Trace {
    double *x, *h1, *h2, *h3, *z, *g4, *d3, *d2, *d1;
};

// mean over the batch of KL(q_i || softmax(z_i)), q_i the i-th target row
// normalised to sum 1, and its gradient with respect to every parameter (the padded input columns of W1 get gradient 0)
static double mlp_grad(const float* params, const float* pos, const float* nrm, size_t n, const float* lo, float S,
                       const float* target, bool bf, double* grad, const Trace* tr) {
    std::vector<double> W[4], B[4];
    unpack(params, bf, W, B);
    const double* b[4] = {B[0].data(), B[1].data(), B[2].data(), B[3].data()};
    std::memset(grad, 0, kParams * sizeof(double));
    double loss = 0.0;
    Fwd f;
    std::vector<double> g4(kOut), d3(kHid), d2(kHid), d1(kHid);
    const double inv_n = 1.0 / (double)n;
    for (size_t s = 0; s < n; ++s) {
        forward_one(W, b, pos + 3 * s, nrm + 3 * s, lo, S, bf, f);
        // q: the target field normalised to sum 1 (any non-negative field is accepted)
        const float* t = target + (size_t)kOut * s;
        double tsum = 0.0;
        for (int c = 0; c < kOut; ++c) tsum += (double)t[c];
        const double inv_t = tsum > 0.0 ? 1.0 / tsum : 0.0;
        for (int c = 0; c < kOut; ++c) {
            const double q = (double)t[c] * inv_t;
            if (q > 0) loss += q * (std::log(q) - std::log(f.p[c]));
            g4[c] = rnd((f.p[c] - q) * inv_n, bf);  // dKL/dz for the batch mean
        }
        // output layer
        for (int o = 0; o < kOut; ++o) {
            for (int i = 0; i < kHid; ++i) grad[kOffW4 + (size_t)o * kHid + i] += g4[o] * f.h3[i];
            grad[kOffB4 + o] += g4[o];
        }
        for (int i = 0; i < kHid; ++i) {
            double s3 = 0.0;
            for (int o = 0; o < kOut; ++o) s3 += g4[o] * W[3][(size_t)o * kHid + i];
            d3[i] = rnd(f.h3[i] > 0 ? s3 : 0.0, bf);
        }
        for (int o = 0; o < kHid; ++o) {
            for (int i = 0; i < kHid; ++i) grad[kOffW3 + (size_t)o * kHid + i] += d3[o] * f.h2[i];
            grad[kOffB3 + o] += d3[o];
        }
        for (int i = 0; i < kHid; ++i) {
            double s2 = 0.0;
            for (int o = 0; o < kHid; ++o) s2 += d3[o] * W[2][(size_t)o * kHid + i];
            d2[i] = rnd(f.h2[i] > 0 ? s2 : 0.0, bf);
        }
        for (int o = 0; o < kHid; ++o) {
            for (int i = 0; i < kHid; ++i) grad[kOffW2 + (size_t)o * kHid + i] += d2[o] * f.h1[i];
            grad[kOffB2 + o] += d2[o];
        }
        for (int i = 0; i < kHid; ++i) {
            double s1 = 0.0;
            for (int o = 0; o < kHid; ++o) s1 += d2[o] * W[1][(size_t)o * kHid + i];
            d1[i] = rnd(f.h1[i] > 0 ? s1 : 0.0, bf);
        }
        for (int o = 0; o < kHid; ++o) {
            for (int i = 0; i < kFeat; ++i) grad[kOffW1 + (size_t)o * kIn + i] += d1[o] * f.x[i];
            grad[kOffB1 + o] += d1[o];
        }
        if (tr) {
            auto put = [s](double* dst, const double* src, int w) {
                if (dst) std::memcpy(dst + (size_t)w * s, src, (size_t)w * sizeof(double));
            };
            put(tr->x, f.x.data(), kIn);
            put(tr->h1, f.h1.data(), kHid);
            put(tr->h2, f.h2.data(), kHid);
            put(tr->h3, f.h3.data(), kHid);
            put(tr->z, f.z.data(), kOut);
            put(tr->g4, g4.data(), kOut);
            put(tr->d3, d3.data(), kHid);
            put(tr->d2, d2.data(), kHid);
            put(tr->d1, d1.data(), kHid);
        }
    }
    return loss * inv_n;
}

}  // namespace orc

extern "C" {

double orc_mlp_grad(const float* params, const float* pos, const float* nrm, size_t n, const float* lo, float S,
                    const float* target, int bf16, double* grad) {
    return orc::mlp_grad(params, pos, nrm, n, lo, S, target, bf16 != 0, grad, nullptr);
}

// orc_mlp_grad that also hands back its per-sample intermediates: input
// features x [n][80], hidden activations h1..h3 [n][64], logits z [n][1024],
// logit gradients g4 [n][1024] and the masked hidden gradients d3, d2, d1
// [n][64]; the arithmetic is orc_mlp_grad's, unchanged
double orc_mlp_grad_trace(const float* params, const float* pos, const float* nrm, size_t n, const float* lo, float S,
                          const float* target, int bf16, double* grad, double* x, double* h1, double* h2, double* h3,
                          double* z, double* g4, double* d3, double* d2, double* d1) {
    const orc::Trace tr{x, h1, h2, h3, z, g4, d3, d2, d1};
    return orc::mlp_grad(params, pos, nrm, n, lo, S, target, bf16 != 0, grad, &tr);
}

// one Adam step (Kingma & Ba 2015) on float32 master weights; t counts from 1
void orc_adam(float* params, double* m, double* v, const double* grad, size_t P, int t, double lr, double b1,
              double b2, double eps) {
    const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
    for (size_t i = 0; i < P; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        params[i] = (float)((double)params[i] - lr * mh / (std::sqrt(vh) + eps));
    }
}

}  // extern "C"
