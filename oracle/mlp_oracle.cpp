// FP64 CPU oracle of the MLP surrogate of the space-point correction --
// TEST INFRASTRUCTURE ONLY.
//
// Per sector, a 3 -> 64 -> 64 -> 3 network with SiLU activations maps the
// normalised measured position (x, v, z) in [-1, 1]^3 to the correction / 10 cm.
// The network's operands (inputs, weights, activations) are BF16 values
// (round to nearest even of the FP32 value); this oracle applies the same
// rounding to the same values and does every sum and product in FP64.  With
// `exact` = 1 it skips the rounding (used to pin the backward pass by finite
// differences).  The paper has no network: it names the location-dependent
// calibration the correction serves (Abstract, Sec. 3).
//
// Parameter vector (FP32 master copy), 4611 values:
//   W1[64][3], b1[64], W2[64][64] (out, in), b2[64], W3[3][64], b3[3].
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

constexpr int H = 64;
constexpr int OW1 = 0, OB1 = 192, OW2 = 256, OB2 = 4352, OW3 = 4416, OB3 = 4608, NP = 4611;

// BF16 round to nearest even (finite inputs)
double bf16(double v, int exact) {
  if (exact) return v;
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) & 0xFFFF0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

double sig(double z) { return 1.0 / (1.0 + std::exp(-z)); }

struct Acts {
  double a0[3], z1[H], a1[H], z2[H], a2[H], o[3];
};

void forward(const float* P, const double* in, int exact, Acts& A) {
  for (int i = 0; i < 3; ++i) A.a0[i] = bf16(in[i], exact);
  for (int j = 0; j < H; ++j) {
    double s = P[OB1 + j];
    for (int i = 0; i < 3; ++i) s += bf16(P[OW1 + 3 * j + i], exact) * A.a0[i];
    A.z1[j] = s;
    A.a1[j] = bf16(s * sig(s), exact);
  }
  for (int j = 0; j < H; ++j) {
    double s = P[OB2 + j];
    for (int i = 0; i < H; ++i) s += bf16(P[OW2 + H * j + i], exact) * A.a1[i];
    A.z2[j] = s;
    A.a2[j] = bf16(s * sig(s), exact);
  }
  for (int c = 0; c < 3; ++c) {
    double s = P[OB3 + c];
    for (int i = 0; i < H; ++i) s += bf16(P[OW3 + H * c + i], exact) * A.a2[i];
    A.o[c] = s;
  }
}

double dsilu(double z) {
  const double s = sig(z);
  return s * (1.0 + z * (1.0 - s));
}

}  // namespace

extern "C" {

// counter-based uniform in [0, 1): splitmix64 (Steele, Lea, Flood 2014) applied
// three times to (seed, a, b) then index k; top 24 bits.
static uint64_t sm64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double orc_counter_uniform(uint64_t seed, uint64_t a, uint64_t b, uint64_t k) {
  const uint64_t h = sm64(sm64(sm64(seed + a) + b) + k);
  return (double)(h >> 40) * (1.0 / 16777216.0);
}

int orc_mlp_nparams() { return NP; }

float orc_bf16(float v) { return (float)bf16(v, 0); }

// out[n][3] = network output (correction / 10 cm) for normalised inputs in[n][3]
void orc_mlp_forward(const float* P, int n, const double* in, int exact, double* out) {
  Acts A;
  for (int b = 0; b < n; ++b) {
    forward(P, in + 3 * b, exact, A);
    for (int c = 0; c < 3; ++c) out[3 * b + c] = A.o[c];
  }
}

// Loss L = (1/n) sum_b sum_c (o_bc - t_bc)^2 and dL/dP (straight through the
// BF16 rounding: products use the rounded values, gradients pass unchanged).
double orc_mlp_grad(const float* P, int n, const double* in, const double* tgt, int exact, double* grad) {
  std::memset(grad, 0, sizeof(double) * NP);
  double loss = 0.0;
  Acts A;
  for (int b = 0; b < n; ++b) {
    forward(P, in + 3 * b, exact, A);
    double go[3];
    for (int c = 0; c < 3; ++c) {
      const double r = A.o[c] - tgt[3 * b + c];
      loss += r * r;
      go[c] = 2.0 * r / n;
    }
    double ga2[H], gz2[H], ga1[H], gz1[H];
    for (int i = 0; i < H; ++i) ga2[i] = 0.0;
    for (int c = 0; c < 3; ++c) {
      grad[OB3 + c] += go[c];
      for (int i = 0; i < H; ++i) {
        grad[OW3 + H * c + i] += go[c] * A.a2[i];
        ga2[i] += bf16(P[OW3 + H * c + i], exact) * go[c];
      }
    }
    for (int j = 0; j < H; ++j) gz2[j] = ga2[j] * dsilu(A.z2[j]);
    for (int i = 0; i < H; ++i) ga1[i] = 0.0;
    for (int j = 0; j < H; ++j) {
      grad[OB2 + j] += gz2[j];
      for (int i = 0; i < H; ++i) {
        grad[OW2 + H * j + i] += gz2[j] * A.a1[i];
        ga1[i] += bf16(P[OW2 + H * j + i], exact) * gz2[j];
      }
    }
    for (int j = 0; j < H; ++j) gz1[j] = ga1[j] * dsilu(A.z1[j]);
    for (int j = 0; j < H; ++j) {
      grad[OB1 + j] += gz1[j];
      for (int i = 0; i < 3; ++i) grad[OW1 + 3 * j + i] += gz1[j] * A.a0[i];
    }
  }
  return loss / n;
}

// One Adam step at step t (1-based) of T with a cosine learning rate
// lr_t = lr * (1 + cos(pi (t - 1) / T)) / 2 (Kingma and Ba 2015, bias-corrected).
void orc_adam(double* w, double* m, double* v, const double* g, int n, int t, int T, double lr, double b1, double b2,
              double eps) {
  const double lrt = lr * 0.5 * (1.0 + std::cos(M_PI * (t - 1) / (double)T));
  for (int i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / (1.0 - std::pow(b1, t));
    const double vh = v[i] / (1.0 - std::pow(b2, t));
    w[i] -= lrt * mh / (std::sqrt(vh) + eps);
  }
}

// Xavier-uniform initial weights of one sector from the counter generator
// (stream a = sector, b = 0x5EED00000000, k = parameter index); biases 0.
void orc_mlp_init(uint64_t seed, int sector, float* P) {
  for (int k = 0; k < NP; ++k) {
    double lim = 0.0;
    if (k < OB1) lim = std::sqrt(6.0 / (3 + H));
    else if (k >= OW2 && k < OB2) lim = std::sqrt(6.0 / (H + H));
    else if (k >= OW3 && k < OB3) lim = std::sqrt(6.0 / (H + 3));
    P[k] = lim > 0.0 ? (float)((2.0 * orc_counter_uniform(seed, (uint64_t)sector, 0x5EED00000000ull, (uint64_t)k) - 1.0) * lim)
                     : 0.0f;
  }
}

// Training batch of one step: sample k uses u_c = uniform(seed, sector, step,
// 3k + c); the normalised input is 2u - 1 (the grid's bounds box), the target
// (0, dy, dz) / 10 cm of the trilinear grid at that point (grid float32
// [nx][ny][nz][3] of this sector, read in index space u_c (n_c - 1)).
void orc_mlp_batch(uint64_t seed, int sector, uint64_t step, int n, const float* grid, int nx, int ny, int nz,
                   double* in, double* tgt) {
  for (int k = 0; k < n; ++k) {
    double u[3];
    for (int c = 0; c < 3; ++c) u[c] = orc_counter_uniform(seed, (uint64_t)sector, step, 3ull * k + c);
    const int dims[3] = {nx, ny, nz};
    int lo[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      const double t = u[a] * (dims[a] - 1);
      int i = (int)std::floor(t);
      if (i > dims[a] - 2) i = dims[a] - 2;
      lo[a] = i;
      f[a] = t - i;
    }
    double acc[2] = {0.0, 0.0};
    for (int cx = 0; cx < 2; ++cx)
      for (int cy = 0; cy < 2; ++cy)
        for (int cz = 0; cz < 2; ++cz) {
          const double w = (cx ? f[0] : 1 - f[0]) * (cy ? f[1] : 1 - f[1]) * (cz ? f[2] : 1 - f[2]);
          const size_t node = ((size_t)(lo[0] + cx) * ny + lo[1] + cy) * nz + lo[2] + cz;
          acc[0] += w * grid[3 * node + 1];
          acc[1] += w * grid[3 * node + 2];
        }
    for (int c = 0; c < 3; ++c) in[3 * k + c] = 2.0 * u[c] - 1.0;
    tgt[3 * k] = 0.0;
    tgt[3 * k + 1] = acc[0] / 10.0;
    tgt[3 * k + 2] = acc[1] / 10.0;
  }
}
}
