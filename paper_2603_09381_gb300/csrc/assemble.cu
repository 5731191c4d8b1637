// Node geometry, plane-wave right-hand sides, self blocks (Kress log split +
// Maue) and gathered off-diagonal entries of the PMCHWT (Omit) system.
//
// Kernel normalisation G = (i/4) H0(k r); with d = x - y, r = |d|:
//   S = (i/4) H0,  D = (ik/4) H1 (n_y.d)/r,  D* = -(ik/4) H1 (n_x.d)/r,
//   N = (ik/4) [k H0 (n_x.d)(n_y.d)/r^2 + H1/r (n_x.n_y - 2 (n_x.d)(n_y.d)/r^2)]
// (paper Sec. 2.1, eqs. slp, dlp, d_slp, d_dlp).  Off-diagonal FP64 entries
// use hankel.cuh; the self blocks call CUDA's j0/j1/y0/y1, and the FP32
// entries of the mixed mode j0f/j1f/y0f/y1f.
#include "assemble.cuh"
#include "hankel.cuh"
#include "prof.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double EULER_C = 0.57721566490153286061;

__device__ __forceinline__ void polar_r(const InclDev& c, double t, double& r, double& dr, double& ddr) {
  if (c.shape == 0) { r = c.prm[0]; dr = 0; ddr = 0; return; }
  if (c.shape == 2) {
    double r0 = c.prm[0], e = c.prm[1], p = c.prm[2];
    double cs, sn; sincos(p * t, &sn, &cs);
    r = r0 * (1 + e * cs); dr = -r0 * e * p * sn; ddr = -r0 * e * p * p * cs; return;
  }
  // fourier: r0 (1 + sum_{m=2..6} a_m cos(m t + phi_m))
  double r0 = c.prm[0];
  double a = 1, b = 0, d = 0;
  for (int i = 0; i < 5; ++i) {
    double m = 2 + i, am = c.prm[1 + i], ph = c.prm[6 + i];
    double cs, sn; sincos(m * t + ph, &sn, &cs);
    a += am * cs; b -= am * m * sn; d -= am * m * m * cs;
  }
  r = r0 * a; dr = r0 * b; ddr = r0 * d;
}

__global__ void k_geom_nodes(const InclDev* __restrict__ inc, NodesDev nd, int total) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  const int j = nd.incl[g];
  const InclDev c = inc[j];
  const int l = g - c.node_off;
  const int n = c.n;
  const double t = 2 * PI * l / n;
  double ct, st; sincos(t, &st, &ct);
  double lx, ly, dx, dy, ddx, ddy;
  if (c.shape == 1) {
    double a = c.prm[0], b = c.prm[1];
    lx = a * ct; ly = b * st; dx = -a * st; dy = b * ct; ddx = -a * ct; ddy = -b * st;
  } else {
    double r, dr, ddr; polar_r(c, t, r, dr, ddr);
    lx = r * ct; ly = r * st;
    dx = dr * ct - r * st; dy = dr * st + r * ct;
    ddx = ddr * ct - 2 * dr * st - r * ct; ddy = ddr * st + 2 * dr * ct - r * st;
  }
  double cr, sr; sincos(c.rot, &sr, &cr);
  double X = c.cx + cr * lx - sr * ly, Y = c.cy + sr * lx + cr * ly;
  double DX = cr * dx - sr * dy, DY = sr * dx + cr * dy;
  double DDX = cr * ddx - sr * ddy, DDY = sr * ddx + cr * ddy;
  double sp = sqrt(DX * DX + DY * DY);
  double nx = DY / sp, ny = -DX / sp;
  nd.x[g] = X; nd.y[g] = Y; nd.nx[g] = nx; nd.ny[g] = ny;
  nd.speed[g] = sp; nd.w[g] = 2 * PI / n * sp;
  nd.curv[g] = (nx * DDX + ny * DDY) / sp;
  // Kress weight R_n(s), s = 2 pi l / n:
  //   -(4 pi/n) sum_{m=1}^{n/2-1} cos(m s)/m - (4 pi/n^2) cos(n s/2)
  double acc = 0;
  for (int m = 1; m < n / 2; ++m) acc += cos(2 * PI * (double)((long long)m * l % n) / n) / m;
  nd.kress[g] = -(4 * PI / n) * acc - (4 * PI / ((double)n * n)) * ((l & 1) ? -1.0 : 1.0);
}

__global__ void k_points_from_nodes(NodesDev nd, PointsDev p, int total) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  p.x[g] = nd.x[g]; p.y[g] = nd.y[g]; p.nx[g] = nd.nx[g]; p.ny[g] = nd.ny[g]; p.w[g] = nd.w[g];
}

__global__ void k_proxy_points(const ProxyBoxDev* __restrict__ box, int nbox, PointsDev p, int total, int off) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nbox;
  while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (box[mid].point_off <= g) lo = mid; else hi = mid; }
  const ProxyBoxDev b = box[lo];
  int s = g - b.point_off;
  double th = 2 * PI * (s + b.phase) / b.p;
  double c, sn; sincos(th, &sn, &c);
  int q = off + g;
  p.x[q] = b.cx + b.R * c; p.y[q] = b.cy + b.R * sn;
  p.nx[q] = c; p.ny[q] = sn; p.w[q] = 2 * PI * b.R / b.p;
}

template <typename C>
__global__ void k_plane_wave(const InclDev* __restrict__ inc, NodesDev nd, int total, double k0,
                             const double* __restrict__ ang, int nrhs, C* F, int ldf) {
  typedef typename real_of<C>::type R;
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (g >= total || r >= nrhs) return;
  const InclDev c = inc[nd.incl[g]];
  const int l = g - c.node_off;
  double ca, sa; sincos(ang[r], &sa, &ca);
  double ph = k0 * (ca * nd.x[g] + sa * nd.y[g]);
  double cp, sp; sincos(ph, &sp, &cp);
  double dn = k0 * (ca * nd.nx[g] + sa * nd.ny[g]);
  // f = [-u^I; -q^I], q^I = (1/eps+) i k0 (d.n) u^I with eps+ = 1
  F[c.row_off + l + (size_t)r * ldf] = mk((R)(-cp), (R)(-sp));
  F[c.row_off + c.n + l + (size_t)r * ldf] = mk((R)(dn * sp), (R)(-dn * cp));
}

// Bessel J0, Y0, J1, Y1 of a positive real argument.
__device__ __forceinline__ void bessel4(double z, double& j0v, double& y0v, double& j1v, double& y1v) {
  j0v = j0(z); y0v = y0(z); j1v = j1(z); y1v = y1(z);
}

// Kress-split S, D, D* of one wavenumber at node pair (i, l) of one curve
// (complex wavenumber allowed); outputs the quadrature-weighted entries.
struct SelfGeo {
  int i, l, n;
  double h, Rw, spi, spl, curv, ndy, ndx, r, logsin;
};

__device__ __forceinline__ void kress_entries(const SelfGeo& q, double2 k, double2& S, double2& D, double2& T) {
  const double PI4 = 4 * PI;
  if (q.i == q.l) {
    // M1 = -|x'|/(4 pi); M2 = [i/4 - C/(2 pi) - ln(k |x'|/2)/(2 pi)] |x'|;  L2 = L2* = (n.x'')/(4 pi |x'|)
    const double M1 = -q.spi / PI4;
    const double2 lg = zlog(make_double2(0.5 * k.x * q.spi, 0.5 * k.y * q.spi));
    const double2 M2 = make_double2((-EULER_C / (2 * PI) - lg.x / (2 * PI)) * q.spi, (0.25 - lg.y / (2 * PI)) * q.spi);
    S = make_double2(q.Rw * M1 + q.h * M2.x, q.h * M2.y);
    const double L2 = q.curv / PI4;
    D = make_double2(q.h * L2, 0);
    T = D;
    return;
  }
  double2 J0, Y0, J1, Y1;
  const double2 z = make_double2(k.x * q.r, k.y * q.r);
  if (k.y == 0) {
    double j0r, y0r, j1r, y1r;
    bessel4(z.x, j0r, y0r, j1r, y1r);
    J0 = make_double2(j0r, 0); Y0 = make_double2(y0r, 0); J1 = make_double2(j1r, 0); Y1 = make_double2(y1r, 0);
  } else {
    bessel_complex(z, J0, Y0, J1, Y1);
  }
  // single layer: M = (i/4) H0 |x'| = (i J0 - Y0)/4 |x'|,  M1 = -(1/4pi) J0 |x'|
  const double2 M = make_double2(-0.25 * Y0.x * q.spl - 0.25 * J0.y * q.spl, 0.25 * J0.x * q.spl - 0.25 * Y0.y * q.spl);
  const double2 M1 = make_double2(-J0.x * q.spl / PI4, -J0.y * q.spl / PI4);
  S = make_double2(q.Rw * M1.x + q.h * (M.x - M1.x * q.logsin), q.Rw * M1.y + q.h * (M.y - M1.y * q.logsin));
  // H1 = J1 + i Y1;  (i k/4) H1 g  and  -(k/4pi) J1 g
  const double2 H1 = make_double2(J1.x - Y1.y, J1.y + Y1.x);
  const double2 ik4 = make_double2(-0.25 * k.y, 0.25 * k.x);
  const double2 kH = zmul(ik4, H1);
  const double2 kJ = zmul(make_double2(k.x / PI4, k.y / PI4), J1);
  {
    const double g = q.ndy * q.spl;          // double layer
    const double2 L = make_double2(kH.x * g, kH.y * g), L1 = make_double2(-kJ.x * g, -kJ.y * g);
    D = make_double2(q.Rw * L1.x + q.h * (L.x - L1.x * q.logsin), q.Rw * L1.y + q.h * (L.y - L1.y * q.logsin));
  }
  {
    const double g = q.ndx * q.spl;          // adjoint: the same with -g
    const double2 L = make_double2(-kH.x * g, -kH.y * g), L1 = make_double2(kJ.x * g, kJ.y * g);
    T = make_double2(q.Rw * L1.x + q.h * (L.x - L1.x * q.logsin), q.Rw * L1.y + q.h * (L.y - L1.y * q.logsin));
  }
}

template <typename C>
__global__ void __launch_bounds__(256) k_self_pointwise(const InclDev* __restrict__ inc, NodesDev nd, double k0,
                                                        C* const* __restrict__ Aptr, const int* __restrict__ ldA,
                                                        C* const* __restrict__ Cptr, int bm) {
  typedef typename real_of<C>::type R;
  const int j = blockIdx.y;
  const InclDev c = inc[j];
  const int n = c.n;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  SelfGeo q;
  q.i = e % n; q.l = e / n; q.n = n;
  const int gi = c.node_off + q.i, gl = c.node_off + q.l;
  q.h = 2 * PI / n;
  q.spl = nd.speed[gl]; q.spi = nd.speed[gi];
  q.curv = nd.curv[gi];
  const double nxi = nd.nx[gi], nyi = nd.ny[gi], nxl = nd.nx[gl], nyl = nd.ny[gl];
  const double nn = nxi * nxl + nyi * nyl;
  q.Rw = nd.kress[c.node_off + (q.i - q.l + n) % n];
  q.r = 0; q.ndy = 0; q.ndx = 0; q.logsin = 0;
  if (q.i != q.l) {
    const double dx = nd.x[gi] - nd.x[gl], dy = nd.y[gi] - nd.y[gl];
    q.r = sqrt(dx * dx + dy * dy);
    q.ndy = (nxl * dx + nyl * dy) / q.r;
    q.ndx = (nxi * dx + nyi * dy) / q.r;
    const double sn = sin(PI * (double)(q.i - q.l) / n);
    q.logsin = log(4 * sn * sn);
  }
  double2 Sp, Dp, Tp, Sm, Dm, Tm;
  kress_entries(q, make_double2(k0, 0), Sp, Dp, Tp);
  const double2 km = make_double2(c.k_in_re, c.k_in_im);
  kress_entries(q, km, Sm, Dm, Tm);
  const double2 em = make_double2(c.eps_in_re, c.eps_in_im);
  C* A = Aptr[j];
  const size_t lda = ldA[j];
  const int i = q.i, l = q.l;
  if (bm) {
    // Burton-Miller (eps+ = 1, alpha = i/k+): [[D+ - I/2 + alpha N+, -S+ - alpha (D*+ + I/2)],
    // [D- + I/2, -eps- S-]]; here the pointwise part of alpha N+ (alpha k+^2 S+ o nn), the
    // Maue part alpha diag(1/|x'|) Dt S0+ Dt follows through the middle factor alpha S0+
    const double half = (i == l) ? 0.5 : 0.0;
    const double2 al = make_double2(0.0, 1.0 / k0);
    const double a0 = k0 * k0 * nn;
    const double2 aN = zmul(al, make_double2(a0 * Sp.x, a0 * Sp.y));
    A[i + (size_t)l * lda] = mk((R)(Dp.x - half + aN.x), (R)(Dp.y + aN.y));
    const double2 aT = zmul(al, make_double2(Tp.x + half, Tp.y));
    A[i + (size_t)(n + l) * lda] = mk((R)(-Sp.x - aT.x), (R)(-Sp.y - aT.y));
    A[n + i + (size_t)l * lda] = mk((R)(Dm.x + half), (R)Dm.y);
    const double2 eS = zmul(em, Sm);
    A[n + i + (size_t)(n + l) * lda] = mk((R)(-eS.x), (R)(-eS.y));
    const double2 aS = zmul(al, make_double2(Sp.x / q.spl, Sp.y / q.spl));
    Cptr[j][i + (size_t)l * n] = mk((R)aS.x, (R)aS.y);
    return;
  }
  // [[-(e+ S+ + e- S-), D+ + D-], [-(D*+ + D*-), k+^2/e+ S+ o nn + k-^2/e- S- o nn (+ Maue part)]]
  const double2 eS = zmul(em, Sm);
  A[i + (size_t)l * lda] = mk((R)(-(Sp.x + eS.x)), (R)(-(Sp.y + eS.y)));
  A[i + (size_t)(n + l) * lda] = mk((R)(Dp.x + Dm.x), (R)(Dp.y + Dm.y));
  A[n + i + (size_t)l * lda] = mk((R)(-(Tp.x + Tm.x)), (R)(-(Tp.y + Tm.y)));
  const double2 k2e = zdiv(zmul(km, km), em);
  const double a0 = k0 * k0 * nn;
  const double2 nS = zmul(make_double2(k2e.x * nn, k2e.y * nn), Sm);
  A[n + i + (size_t)(n + l) * lda] = mk((R)(a0 * Sp.x + nS.x), (R)(a0 * Sp.y + nS.y));
  // Maue middle factor: S0+/e+ + S0-/e-, S0 = S / |x'(tau)|
  const double2 Se = zdiv(Sm, em);
  C* Cm = Cptr[j];
  Cm[i + (size_t)l * n] = mk((R)((Sp.x + Se.x) / q.spl), (R)((Sp.y + Se.y) / q.spl));
}

template <typename C>
__global__ void k_diff_matrix(int n, C* Dt) {
  typedef typename real_of<C>::type R;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int i = e % n, j = e / n;
  double v = 0;
  if (i != j) {
    int d = i - j;
    v = 0.5 * ((d & 1) ? -1.0 : 1.0) / tan(PI * (double)d / n);
  }
  Dt[e] = mk((R)v, (R)0);
}

template <typename C>
__global__ void k_scaled_diff(const InclDev* __restrict__ inc, NodesDev nd, C* const* __restrict__ out) {
  typedef typename real_of<C>::type R;
  const int j = blockIdx.y;
  const InclDev c = inc[j];
  const int n = c.n;
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * n) return;
  int i = e % n, l = e / n;
  double v = 0;
  if (i != l) {
    int d = i - l;
    v = 0.5 * ((d & 1) ? -1.0 : 1.0) / tan(PI * (double)d / n) / nd.speed[c.node_off + i];
  }
  out[j][e] = mk((R)v, (R)0);
}

// Omit off-diagonal entry between a target (row group rg) and a source (column group cg).
template <typename C>
__device__ __forceinline__ C omit_entry(const PointsDev& P, int t, int s, double k) {
  typedef typename real_of<C>::type R;
  const int pt = t >> 1, rg = t & 1, ps = s >> 1, cg = s & 1;
  const double dx = P.x[pt] - P.x[ps], dy = P.y[pt] - P.y[ps];
  const double r2 = dx * dx + dy * dy;
  if (!(r2 > 0)) return czero<C>();
  const double r = sqrt(r2);
  const double z = k * r;
  const double w = P.w[ps];
  double J0, Y0, J1, Y1;
  if (z < HK_ZA) {                  // near entries: only the Bessel pair the entry needs
    if (rg == 0 && cg == 0) return mk((R)(0.25 * y0(z) * w), (R)(-0.25 * j0(z) * w));
    J1 = j1(z); Y1 = y1(z);
    if (rg == 1 && cg == 1) { J0 = j0(z); Y0 = y0(z); } else { J0 = 0; Y0 = 0; }
  } else {
    hankel01(z, J0, Y0, J1, Y1);
  }
  if (rg == 0 && cg == 0)           // -eps+ S = -(i/4) H0 w
    return mk((R)(0.25 * Y0 * w), (R)(-0.25 * J0 * w));
  if (rg == 0) {                    // D = (ik/4) H1 (n_y.d)/r w
    double g = (P.nx[ps] * dx + P.ny[ps] * dy) / r * 0.25 * k * w;
    return mk((R)(-Y1 * g), (R)(J1 * g));
  }
  if (cg == 0) {                    // -D* = (ik/4) H1 (n_x.d)/r w
    double g = (P.nx[pt] * dx + P.ny[pt] * dy) / r * 0.25 * k * w;
    return mk((R)(-Y1 * g), (R)(J1 * g));
  }
  // N/eps+ = (ik/4) [k H0 a b + H1/r (nn - 2 a b)] w,  a = n_x.d/r, b = n_y.d/r
  const double a = (P.nx[pt] * dx + P.ny[pt] * dy) / r, b = (P.nx[ps] * dx + P.ny[ps] * dy) / r;
  const double nn = P.nx[pt] * P.nx[ps] + P.ny[pt] * P.ny[ps];
  const double c0 = k * a * b, c1 = (nn - 2 * a * b) / r;
  const double Hre = c0 * J0 + c1 * J1, Him = c0 * Y0 + c1 * Y1;   // k H0 ab + H1/r (...)
  const double f = 0.25 * k * w;
  return mk((R)(-Him * f), (R)(Hre * f));
}

// Single-precision entry (the FP32 factorization of the mixed-precision mode).
template <>
__device__ __forceinline__ float2 omit_entry<float2>(const PointsDev& P, int t, int s, double k) {
  const int pt = t >> 1, rg = t & 1, ps = s >> 1, cg = s & 1;
  const float dx = (float)(P.x[pt] - P.x[ps]), dy = (float)(P.y[pt] - P.y[ps]);
  const float r2 = dx * dx + dy * dy;
  if (!(r2 > 0.f)) return make_float2(0.f, 0.f);
  const float r = sqrtf(r2);
  const float kf = (float)k;
  const float z = kf * r;
  const float w = (float)P.w[ps];
  const float ntx = (float)P.nx[pt], nty = (float)P.ny[pt], nsx = (float)P.nx[ps], nsy = (float)P.ny[ps];
  if (rg == 0 && cg == 0) return make_float2(0.25f * y0f(z) * w, -0.25f * j0f(z) * w);
  const float J1 = j1f(z), Y1 = y1f(z);
  if (rg == 0) {
    float g = (nsx * dx + nsy * dy) / r * 0.25f * kf * w;
    return make_float2(-Y1 * g, J1 * g);
  }
  if (cg == 0) {
    float g = (ntx * dx + nty * dy) / r * 0.25f * kf * w;
    return make_float2(-Y1 * g, J1 * g);
  }
  const float J0 = j0f(z), Y0 = y0f(z);
  const float a = (ntx * dx + nty * dy) / r, b = (nsx * dx + nsy * dy) / r;
  const float nn = ntx * nsx + nty * nsy;
  const float c0 = kf * a * b, c1 = (nn - 2.f * a * b) / r;
  const float Hre = c0 * J0 + c1 * J1, Him = c0 * Y0 + c1 * Y1;
  const float f = 0.25f * kf * w;
  return make_float2(-Him * f, Hre * f);
}

// The four trapezoid-rule kernels S, D, D*, N (times the source weight) between
// point t and point s for wavenumber k (G = (i/4) H0(k r)).
__device__ __forceinline__ void kernels4(const PointsDev& P, int pt, int ps, double k, double2& S, double2& D,
                                         double2& Ds, double2& N) {
  const double dx = P.x[pt] - P.x[ps], dy = P.y[pt] - P.y[ps];
  const double r = sqrt(dx * dx + dy * dy);
  const double z = k * r, w = P.w[ps];
  double J0, Y0, J1, Y1;
  if (z < HK_ZA) { J0 = j0(z); Y0 = y0(z); J1 = j1(z); Y1 = y1(z); }
  else hankel01(z, J0, Y0, J1, Y1);
  const double a = (P.nx[pt] * dx + P.ny[pt] * dy) / r, b = (P.nx[ps] * dx + P.ny[ps] * dy) / r;
  const double nn = P.nx[pt] * P.nx[ps] + P.ny[pt] * P.ny[ps];
  const double f = 0.25 * k * w;
  S = make_double2(-0.25 * Y0 * w, 0.25 * J0 * w);       // (i/4) H0 w
  D = make_double2(-Y1 * b * f, J1 * b * f);               // (ik/4) H1 b w
  Ds = make_double2(Y1 * a * f, -J1 * a * f);              // -(ik/4) H1 a w
  const double c0 = k * a * b, c1 = (nn - 2 * a * b) / r;
  N = make_double2(-(c0 * Y0 + c1 * Y1) * f, (c0 * J0 + c1 * J1) * f);
}

// Entry of the PMCHWT (All), Burton-Miller or interior-family systems (FP64).
__device__ double2 form_entry(const PointsDev& P, int t, int s, const GatherProb<double2>& g, double k) {
  const int pt = t >> 1, rg = t & 1, ps = s >> 1, cg = s & 1;
  const double dx = P.x[pt] - P.x[ps], dy = P.y[pt] - P.y[ps];
  if (!(dx * dx + dy * dy > 0)) return make_double2(0, 0);
  auto omit_like = [&](double kk, double eps) {
    double2 S, D, Ds, N;
    kernels4(P, pt, ps, kk, S, D, Ds, N);
    if (rg == 0) return cg == 0 ? make_double2(-eps * S.x, -eps * S.y) : D;
    return cg == 0 ? make_double2(-Ds.x, -Ds.y) : make_double2(N.x / eps, N.y / eps);
  };
  if (g.mode == GATHER_INTERIOR) return omit_like(g.k_in, g.eps_in);
  if (g.mode == GATHER_ALL) {
    const double2 e = omit_like(k, 1.0), i2 = omit_like(g.k_in, g.eps_in);
    return make_double2(e.x + i2.x, e.y + i2.y);
  }
  // Burton-Miller
  if (rg == 1) {
    if (g.mode == GATHER_BM_SIMPLIFIED) return make_double2(0, 0);
    double2 S, D, Ds, N;
    kernels4(P, pt, ps, g.k_in, S, D, Ds, N);
    return cg == 0 ? D : make_double2(-g.eps_in * S.x, -g.eps_in * S.y);
  }
  double2 S, D, Ds, N;
  kernels4(P, pt, ps, k, S, D, Ds, N);
  const double ia = 1.0 / k;   // alpha = i / k
  if (cg == 0) return make_double2(D.x - ia * N.y, D.y + ia * N.x);            // D + alpha N
  return make_double2(-(S.x - ia * Ds.y), -(S.y + ia * Ds.x));                 // -(S + alpha D*)
}

template <typename C>
__device__ __forceinline__ C gather_entry(const PointsDev& P, int t, int s, const GatherProb<C>& g, double k);
template <>
__device__ __forceinline__ double2 gather_entry<double2>(const PointsDev& P, int t, int s,
                                                         const GatherProb<double2>& g, double k) {
  return g.mode == GATHER_OMIT ? omit_entry<double2>(P, t, s, k) : form_entry(P, t, s, g, k);
}
template <>
__device__ __forceinline__ float2 gather_entry<float2>(const PointsDev& P, int t, int s, const GatherProb<float2>& g,
                                                       double k) {
  return omit_entry<float2>(P, t, s, k);   // the complex64 path is PMCHWT (Omit) only
}

template <typename C>
__global__ void __launch_bounds__(256) k_gather(const GatherProb<C>* __restrict__ prob, const int* __restrict__ tile_off,
                                                int nprob, PointsDev P, double k) {
  int t = blockIdx.x;
  int lo = 0, hi = nprob;
  while (hi - lo > 1) { int mid = (lo + hi) >> 1; if (tile_off[mid] <= t) lo = mid; else hi = mid; }
  const GatherProb<C> g = prob[lo];
  int local = t - tile_off[lo];
  int tiles_m = (g.M + 31) / 32;
  int i = (local % tiles_m) * 32 + (threadIdx.x & 31);
  int j = (local / tiles_m) * 8 + (threadIdx.x >> 5);
  if (i >= g.M || j >= g.N) return;
  int tc = g.trans ? g.tgt[j] : g.tgt[i];
  int sc = g.trans ? g.src[i] : g.src[j];
  g.out[i + (size_t)j * g.ld] = gather_entry<C>(P, tc, sc, g, g.k != 0.0 ? g.k : k);
}

}  // namespace

void geom_nodes(const InclDev* d_inc, NodesDev nodes, int total, const InclDev*, cudaStream_t st) {
  if (total <= 0) return;
  k_geom_nodes<<<(total + 127) / 128, 128, 0, st>>>(d_inc, nodes, total);
  pm_launch_count_add(1);
}

void geom_points_from_nodes(NodesDev nodes, PointsDev pts, int total, cudaStream_t st) {
  if (total <= 0) return;
  k_points_from_nodes<<<(total + 255) / 256, 256, 0, st>>>(nodes, pts, total);
  pm_launch_count_add(1);
}

void geom_proxy_points(const ProxyBoxDev* d_box, int nbox, PointsDev pts, int total, int off, cudaStream_t st) {
  if (total <= 0 || nbox <= 0) return;
  k_proxy_points<<<(total + 255) / 256, 256, 0, st>>>(d_box, nbox, pts, total, off);
  pm_launch_count_add(1);
}

template <typename C>
void plane_wave_rhs(const InclDev* d_inc, NodesDev nodes, int total, double k0, const double* d_ang, int nrhs,
                    C* F, int ldf, cudaStream_t st) {
  if (total <= 0 || nrhs <= 0) return;
  dim3 g((total + 255) / 256, nrhs);
  k_plane_wave<C><<<g, 256, 0, st>>>(d_inc, nodes, total, k0, d_ang, nrhs, F, ldf);
  pm_launch_count_add(1);
}

template <typename C>
void self_pointwise(const InclDev* d_inc, int m, int maxn, NodesDev nodes, double k0, C* const* d_A,
                    const int* d_lda, C* const* d_Cm, cudaStream_t st, int bm) {
  if (m <= 0) return;
  dim3 g((maxn * maxn + 255) / 256, m);
  KPROF_BEGIN(st);
  k_self_pointwise<C><<<g, 256, 0, st>>>(d_inc, nodes, k0, d_A, d_lda, d_Cm, bm);
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("self_pointwise", "self_pointwise32"), 0.0);
}

__global__ void k_round_blocks(const double2* const* __restrict__ src, float2* const* __restrict__ dst,
                               const int* __restrict__ n) {
  const int b = blockIdx.y, m = n[b];
  const double2* sb = src[b];
  float2* db = dst[b];
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m * m; e += gridDim.x * blockDim.x)
    db[e] = make_float2((float)sb[e].x, (float)sb[e].y);
}

void round_blocks(const double2* const* d_src, float2* const* d_dst, const int* d_n, int nblk, int maxn,
                  cudaStream_t st) {
  if (nblk <= 0 || maxn <= 0) return;
  k_round_blocks<<<dim3(std::min(64, (maxn * maxn + 255) / 256), nblk), 256, 0, st>>>(d_src, d_dst, d_n);
  pm_launch_count_add(1);
}

template <typename C>
void diff_matrices(int n, C* Dt, cudaStream_t st) {
  k_diff_matrix<C><<<(n * n + 255) / 256, 256, 0, st>>>(n, Dt);
  pm_launch_count_add(1);
}

template <typename C>
void scaled_diff(const InclDev* d_inc, int m, int maxn, NodesDev nodes, C* const* d_DtS, cudaStream_t st) {
  if (m <= 0) return;
  dim3 g((maxn * maxn + 255) / 256, m);
  k_scaled_diff<C><<<g, 256, 0, st>>>(d_inc, nodes, d_DtS);
  pm_launch_count_add(1);
}

template <typename C>
void gather_assemble(const GatherProb<C>* d_prob, const int* d_tile_off, int nprob, int total_tiles,
                     PointsDev pts, double k0, cudaStream_t st) {
  if (nprob <= 0 || total_tiles <= 0) return;
  KPROF_BEGIN(st);
  k_gather<C><<<total_tiles, 256, 0, st>>>(d_prob, d_tile_off, nprob, pts, k0);
  pm_launch_count_add(1);
  KPROF_END(st, kname<C>("gather_entries", "gather_entries32"), 0.0);
}

template void plane_wave_rhs<double2>(const InclDev*, NodesDev, int, double, const double*, int, double2*, int, cudaStream_t);
template void self_pointwise<double2>(const InclDev*, int, int, NodesDev, double, double2* const*, const int*,
                                      double2* const*, cudaStream_t, int);
template void diff_matrices<double2>(int, double2*, cudaStream_t);
template void scaled_diff<double2>(const InclDev*, int, int, NodesDev, double2* const*, cudaStream_t);
template void gather_assemble<double2>(const GatherProb<double2>*, const int*, int, int, PointsDev, double, cudaStream_t);

template void self_pointwise<float2>(const InclDev*, int, int, NodesDev, double, float2* const*, const int*,
                                     float2* const*, cudaStream_t, int);
template void diff_matrices<float2>(int, float2*, cudaStream_t);
template void scaled_diff<float2>(const InclDev*, int, int, NodesDev, float2* const*, cudaStream_t);
template void gather_assemble<float2>(const GatherProb<float2>*, const int*, int, int, PointsDev, double, cudaStream_t);
