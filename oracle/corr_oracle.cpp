// FP64 CPU oracle of the space-point corrections -- TEST INFRASTRUCTURE ONLY.
//
// The paper names location-dependent calibration as a condition of the online
// reconstruction (Abstract) and online calibration in the synchronous phase
// (Sec. 3).  The correction here is a per-sector grid of (dx, dy, dz) shifts at
// distorted-space nodes, read by trilinear interpolation (its plain
// definition); the pad row fixes x, so only dy and dz are applied.
#include <cmath>
#include <cstdint>

extern "C" {

// grid: float32 [S][nx][ny][nz][3] over axes (x, v = y / (x tan_half), z);
// bounds: float32 [S][6] = (x0, x1, v0, v1, z0, z1).  Points outside the grid
// use the nearest edge cell (coordinates clamped).  x: pad-row radius.
void orc_trilinear(const float* grid, const float* bounds, int nx, int ny, int nz, double tan_half, int n,
                   const int32_t* sector, const double* x, const double* y, const double* z, double* out_dy,
                   double* out_dz) {
  for (int i = 0; i < n; ++i) {
    const int s = sector[i];
    const float* B = bounds + 6 * (size_t)s;
    const double v = y[i] / (x[i] * tan_half);
    double u[3] = {(x[i] - B[0]) / (B[1] - B[0]) * (nx - 1), (v - B[2]) / (B[3] - B[2]) * (ny - 1),
                   (z[i] - B[4]) / (B[5] - B[4]) * (nz - 1)};
    const int dims[3] = {nx, ny, nz};
    int lo[3];
    double f[3];
    for (int a = 0; a < 3; ++a) {
      double t = u[a];
      if (t < 0.0) t = 0.0;
      if (t > dims[a] - 1) t = dims[a] - 1;
      int k = (int)std::floor(t);
      if (k > dims[a] - 2) k = dims[a] - 2;
      lo[a] = k;
      f[a] = t - k;
    }
    double acc[2] = {0.0, 0.0};
    for (int cx = 0; cx < 2; ++cx)
      for (int cy = 0; cy < 2; ++cy)
        for (int cz = 0; cz < 2; ++cz) {
          const double w = (cx ? f[0] : 1.0 - f[0]) * (cy ? f[1] : 1.0 - f[1]) * (cz ? f[2] : 1.0 - f[2]);
          const size_t node = (((size_t)s * nx + lo[0] + cx) * ny + lo[1] + cy) * nz + lo[2] + cz;
          acc[0] += w * grid[3 * node + 1];
          acc[1] += w * grid[3 * node + 2];
        }
    out_dy[i] = acc[0];
    out_dz[i] = acc[1];
  }
}
}
