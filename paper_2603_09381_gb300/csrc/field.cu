// Off-boundary fields from a boundary solution (see field.cuh).  One CTA per
// (evaluation point or direction, right-hand side) sums the trapezoid rule
// over every node in a fixed order (block-wide reduction), so results are
// reproducible; the far field needs one sincos per term, the near field one
// Hankel pair.
#include "field.cuh"
#include "hankel.cuh"
#include "prof.cuh"

namespace {

constexpr int FT = 256;

__device__ __forceinline__ double2 block_sum2(double2 v, double2* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double2 t = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int w = 0; w < FT / 32; ++w) { t.x += sh[w].x; t.y += sh[w].y; }
  return t;
}

// q and u of node i: phi[row_off + l] and phi[row_off + n + l], l = i - node_off
__device__ __forceinline__ void qu_of(const InclDev* inc, const int* incl, const double2* phi, int i, double2& q,
                                      double2& u) {
  const InclDev d = inc[incl[i]];
  const int l = i - d.node_off;
  q = phi[d.row_off + l];
  u = phi[d.row_off + d.n + l];
}

__global__ void __launch_bounds__(FT) k_far_field(const InclDev* __restrict__ inc, NodesDev nd, int total, double k,
                                                  const double2* __restrict__ phi, int ldphi,
                                                  const double* __restrict__ ang, int ndir, double2* out) {
  __shared__ double2 sh[FT / 32];
  const int dir = blockIdx.x, c = blockIdx.y;
  double sa, ca;
  sincos(ang[dir], &sa, &ca);
  const double2* ph = phi + (size_t)c * ldphi;
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < total; i += FT) {
    double2 q, u;
    qu_of(inc, nd.incl, ph, i, q, u);
    double s, co;
    sincos(-k * (ca * nd.x[i] + sa * nd.y[i]), &s, &co);      // e^{-i k xhat.y}
    const double kn = k * (ca * nd.nx[i] + sa * nd.ny[i]);
    // -i k (xhat.n) u - q  (eps+ = 1)
    const double tx = kn * u.y - q.x, ty = -kn * u.x - q.y;
    const double w = nd.w[i];
    acc.x += w * (co * tx - s * ty);
    acc.y += w * (co * ty + s * tx);
  }
  const double2 t = block_sum2(acc, sh);
  if (threadIdx.x == 0) {
    // gamma = (i/4) sqrt(2/(pi k)) e^{-i pi/4} = (sqrt(2/(pi k)) / 4) e^{i pi/4}
    const double gm = 0.25 * sqrt(2.0 / (3.141592653589793 * k)) * 0.7071067811865476;
    out[dir + (size_t)c * ndir] = make_double2(gm * (t.x - t.y), gm * (t.x + t.y));
  }
}

__global__ void __launch_bounds__(FT) k_scattered(const InclDev* __restrict__ inc, NodesDev nd, int total, double k,
                                                  const double2* __restrict__ phi, int ldphi,
                                                  const double* __restrict__ xy, int npts, double2* out) {
  __shared__ double2 sh[FT / 32];
  const int p = blockIdx.x, c = blockIdx.y;
  const double px = xy[2 * p], py = xy[2 * p + 1];
  const double2* ph = phi + (size_t)c * ldphi;
  double2 acc = make_double2(0, 0);
  for (int i = threadIdx.x; i < total; i += FT) {
    double2 q, u;
    qu_of(inc, nd.incl, ph, i, q, u);
    const double dx = px - nd.x[i], dy = py - nd.y[i];
    const double r = sqrt(dx * dx + dy * dy);
    const double z = k * r;
    double J0, Y0, J1, Y1;
    if (z < HK_ZA) { J0 = j0(z); Y0 = y0(z); J1 = j1(z); Y1 = y1(z); }
    else hankel01(z, J0, Y0, J1, Y1);
    const double b = (nd.nx[i] * dx + nd.ny[i] * dy) / r;
    // G = (i/4) H0 = (-Y0 + i J0)/4;  dG/dn_y = (i k/4) H1 b = k b (-Y1 + i J1)/4
    const double gx = -0.25 * Y0, gy = 0.25 * J0;
    const double dx2 = -0.25 * k * b * Y1, dy2 = 0.25 * k * b * J1;
    const double w = nd.w[i];
    acc.x += w * ((dx2 * u.x - dy2 * u.y) - (gx * q.x - gy * q.y));
    acc.y += w * ((dx2 * u.y + dy2 * u.x) - (gx * q.y + gy * q.x));
  }
  const double2 t = block_sum2(acc, sh);
  if (threadIdx.x == 0) out[p + (size_t)c * npts] = t;
}

}  // namespace

void far_field(const InclDev* d_inc, NodesDev nodes, int total, double k0, const double2* phi, int ldphi, int nrhs,
               const double* d_angles, int ndir, double2* out, cudaStream_t st) {
  if (ndir <= 0 || nrhs <= 0) return;
  k_far_field<<<dim3(ndir, nrhs), FT, 0, st>>>(d_inc, nodes, total, k0, phi, ldphi, d_angles, ndir, out);
  pm_launch_count_add(1);
}

void scattered_field(const InclDev* d_inc, NodesDev nodes, int total, double k0, const double2* phi, int ldphi,
                     int nrhs, const double* d_xy, int npts, double2* out, cudaStream_t st) {
  if (npts <= 0 || nrhs <= 0) return;
  k_scattered<<<dim3(npts, nrhs), FT, 0, st>>>(d_inc, nodes, total, k0, phi, ldphi, d_xy, npts, out);
  pm_launch_count_add(1);
}
