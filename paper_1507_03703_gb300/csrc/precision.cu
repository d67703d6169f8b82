// The all-FP64 evaluation path: the energy components and forces of stored configurations with
// every operation in FP64, on FP64 lattices and FP64 parameters.  It is the FP64 arm of the
// precision study of the FP32 path (grid interaction, "Thermodynamic Cycle"; the ligand force
// field; the restraint, Eq. (binding_site); the state weights, Eq. (protocol)).  One thread
// evaluates one configuration; throughput is not its purpose, and GB300's FP64 rate is a small
// fraction of its FP32 rate.
#include <math.h>

#include "internal.cuh"

namespace algdock {
namespace {

struct V3 {
  double x, y, z;
};
__device__ inline V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ inline V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ inline V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ inline double dot3(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline V3 cross3(V3 a, V3 b) { return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

// Per-configuration views: positions (converted once to FP64 in the force array's slot) and the
// force accumulator, both [na][3] in global memory owned by this thread.
struct Conf {
  const float* x;
  double* f;  // may be null (energies only)
  __device__ V3 pos(int i) const { return V3{(double)x[3 * i], (double)x[3 * i + 1], (double)x[3 * i + 2]}; }
  __device__ void add(int i, V3 v) const {
    if (!f) return;
    f[3 * i] += v.x;
    f[3 * i + 1] += v.y;
    f[3 * i + 2] += v.z;
  }
};

// Trilinear value and gradient of lattice channel ch at p; coordinates outside the lattice are
// clamped to it, and the gradient along a clamped axis is zero.
struct Interp {
  int64_t b;
  double t[3];
  bool in[3];
};
__device__ inline Interp locate(const GridDev64& G, V3 p) {
  Interp I;
  const double o[3] = {G.ox, G.oy, G.oz}, q[3] = {p.x, p.y, p.z};
  const int n[3] = {G.nx, G.ny, G.nz};
  int c[3];
  for (int d = 0; d < 3; ++d) {
    double u = (q[d] - o[d]) / G.h;
    I.in[d] = true;
    if (!(u >= 0.0)) {
      u = 0.0;
      I.in[d] = false;
    }
    if (u > (double)(n[d] - 1)) {
      u = (double)(n[d] - 1);
      I.in[d] = false;
    }
    int ci = (int)floor(u);
    if (ci > n[d] - 2) ci = n[d] - 2;
    c[d] = ci;
    I.t[d] = u - ci;
  }
  I.b = ((int64_t)c[2] * G.ny + c[1]) * G.nx + c[0];
  return I;
}

template <typename Get>
__device__ inline double trilinear(const GridDev64& G, const Interp& I, Get get, V3* grad) {
  const int64_t sy = G.nx, sz = (int64_t)G.nx * G.ny;
  double v = 0.0, gx = 0.0, gy = 0.0, gz = 0.0;
  for (int e = 0; e < 2; ++e)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const double node = get(I.b + e * sz + b * sy + a);
        const double wx = a ? I.t[0] : 1.0 - I.t[0], wy = b ? I.t[1] : 1.0 - I.t[1],
                     wz = e ? I.t[2] : 1.0 - I.t[2];
        const double dx = a ? 1.0 : -1.0, dy = b ? 1.0 : -1.0, dz = e ? 1.0 : -1.0;
        v += wx * wy * wz * node;
        gx += dx * wy * wz * node;
        gy += wx * dy * wz * node;
        gz += wx * wy * dz * node;
      }
  *grad = V3{I.in[0] ? gx / G.h : 0.0, I.in[1] ? gy / G.h : 0.0, I.in[2] ? gz / G.h : 0.0};
  return v;
}

__global__ void __launch_bounds__(128) eval64_kernel(int64_t N, Lig64 L, const double* __restrict__ P, GridDev64 G,
                                                    const StateDev* __restrict__ states, int n_states,
                                                    const int32_t* __restrict__ state_of, const float* __restrict__ x,
                                                    double* force, double* comps) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int na = L.na;
  double w_sg = 0.0, w_g = 0.0;
  if (state_of) {
    const int k = state_of[n];
    if ((unsigned)k < (unsigned)n_states) {
      w_sg = states[k].w_sg;
      w_g = states[k].w_g;
    }
  }
  Conf cf{x + n * na * 3, force ? force + n * na * 3 : nullptr};
  if (cf.f)
    for (int i = 0; i < 3 * na; ++i) cf.f[i] = 0.0;
  const double* atom = P + L.off_atom;
  double e_lig = 0.0;
  // bonds: k (r - r0)^2
  for (int t = 0; t < L.nb; ++t) {
    const double* b = P + L.off_bond + 4 * t;
    const int i = (int)b[0], j = (int)b[1];
    const V3 d = cf.pos(i) - cf.pos(j);
    const double r = sqrt(dot3(d, d));
    const double dr = r - b[3];
    e_lig += b[2] * dr * dr;
    const V3 fi = (-2.0 * b[2] * dr / r) * d;
    cf.add(i, fi);
    cf.add(j, -1.0 * fi);
  }
  // angles: k (theta - theta0)^2, theta at the middle atom
  for (int t = 0; t < L.nang; ++t) {
    const double* a = P + L.off_ang + 5 * t;
    const int i = (int)a[0], j = (int)a[1], k = (int)a[2];
    const V3 u = cf.pos(i) - cf.pos(j), w = cf.pos(k) - cf.pos(j);
    const double lu2 = dot3(u, u), lw2 = dot3(w, w), luw = sqrt(lu2 * lw2);
    const double c = fmin(1.0, fmax(-1.0, dot3(u, w) / luw));
    const double dth = acos(c) - a[4];
    e_lig += a[3] * dth * dth;
    // d theta / d u = -(w / luw - c u / lu2) / sin(theta)
    const double coef = 2.0 * a[3] * dth / sqrt(fmax(1.0 - c * c, 1e-30));
    const V3 fi = coef * ((1.0 / luw) * w - (c / lu2) * u);
    const V3 fk = coef * ((1.0 / luw) * u - (c / lw2) * w);
    cf.add(i, fi);
    cf.add(k, fk);
    cf.add(j, -1.0 * (fi + fk));
  }
  // torsions: sum_n V_n/2 (1 + cos(n phi - gamma_n))
  for (int t = 0; t < L.ntor; ++t) {
    const double* q = P + L.off_tor + 10 * t;
    const int i = (int)q[0], j = (int)q[1], k = (int)q[2], l = (int)q[3];
    const V3 b1 = cf.pos(j) - cf.pos(i), b2 = cf.pos(k) - cf.pos(j), b3 = cf.pos(l) - cf.pos(k);
    const V3 n1 = cross3(b1, b2), n2 = cross3(b2, b3);
    const double lb2 = sqrt(dot3(b2, b2));
    const double n1s = fmax(dot3(n1, n1), 1e-60), n2s = fmax(dot3(n2, n2), 1e-60);
    const double phi = atan2(lb2 * dot3(b1, n2), dot3(n1, n2));
    double dE = 0.0;
    for (int m = 1; m <= 3; ++m) {
      const double arg = m * phi - q[6 + m];
      e_lig += q[3 + m] * (1.0 + cos(arg));
      dE -= q[3 + m] * m * sin(arg);
    }
    // forces: F_i = (dE lb2 / |n1|^2) n1, F_l = -(dE lb2 / |n2|^2) n2, and the middle atoms keep
    // the total force and torque zero
    const V3 fi = (dE * lb2 / n1s) * n1, fl = (-dE * lb2 / n2s) * n2;
    const double p = dot3(b1, b2) / (lb2 * lb2), r = dot3(b3, b2) / (lb2 * lb2);
    cf.add(i, fi);
    cf.add(l, fl);
    cf.add(j, (-(1.0 + p)) * fi + r * fl);
    cf.add(k, p * fi + (-(1.0 + r)) * fl);
  }
  // nonbonded pairs beyond 1-3: Lorentz-Berthelot Lennard-Jones and Coulomb, 1-4 scaled
  for (int i = 0; i < na; ++i)
    for (int j = i + 1; j < na; ++j) {
      const int ty = (int)P[L.off_ptype + (int64_t)j * na + i];
      if (ty == 2) continue;
      const double s_lj = ty == 1 ? 0.5 : 1.0, s_el = ty == 1 ? 1.0 / 1.2 : 1.0;
      const double* ai = atom + 6 * i;
      const double* aj = atom + 6 * j;
      const V3 d = cf.pos(i) - cf.pos(j);
      const double r2 = dot3(d, d), r = sqrt(r2);
      const double R = ai[4] + aj[4], eps = ai[5] * aj[5];
      const double s2 = R * R / r2, s6 = s2 * s2 * s2;
      const double elj = s_lj * eps * (s6 * s6 - 2.0 * s6);
      const double eel = s_el * kCoulomb * ai[1] * aj[1] / r;
      e_lig += elj + eel;
      // -dE/dr / r
      const double fr = (s_lj * eps * 12.0 * (s6 * s6 - s6) + eel) / r2;
      cf.add(i, fr * d);
      cf.add(j, (-fr) * d);
    }
  // restraint on the centre of mass
  V3 com{0.0, 0.0, 0.0};
  for (int i = 0; i < na; ++i) com = com + atom[6 * i] * cf.pos(i);
  com = (1.0 / L.total_mass) * com;
  const V3 dc = com - V3{L.site[0], L.site[1], L.site[2]};
  const double d = sqrt(dot3(dc, dc));
  double e_rest = 0.0;
  if (d > L.d0) {
    const double ex = d - L.d0;
    e_rest = 0.5 * L.k_rest * ex * ex;
    const double c = -L.k_rest * ex / (d * L.total_mass);
    for (int i = 0; i < na; ++i) cf.add(i, (c * atom[6 * i]) * dc);
  } else if (!(d <= L.d0)) {
    e_rest = d;  // NaN centre of mass
  }
  // grid terms: hard Psi_g = sA r^4 + sB a + q e, soft Psi_sg = sA sr^4 + q se
  double psi_g = 0.0, psi_sg = 0.0;
  for (int i = 0; i < na; ++i) {
    const double* ai = atom + 6 * i;
    const Interp I = locate(G, cf.pos(i));
    V3 gr, ga, ge, gsr, gse;
    const double r = trilinear(G, I, [&](int64_t m) { return G.hard[m].r; }, &gr);
    const double la = trilinear(G, I, [&](int64_t m) { return G.hard[m].a; }, &ga);
    const double le = trilinear(G, I, [&](int64_t m) { return G.hard[m].e; }, &ge);
    const double sr = trilinear(G, I, [&](int64_t m) { return G.soft[m].r; }, &gsr);
    const double se = trilinear(G, I, [&](int64_t m) { return G.soft[m].e; }, &gse);
    psi_g += ai[2] * (r * r) * (r * r) + ai[3] * la + ai[1] * le;
    psi_sg += ai[2] * (sr * sr) * (sr * sr) + ai[1] * se;
    if (cf.f) {
      const V3 dg = (4.0 * ai[2] * r * r * r) * gr + ai[3] * ga + ai[1] * ge;
      const V3 dsg = (4.0 * ai[2] * sr * sr * sr) * gsr + ai[1] * gse;
      cf.add(i, (-w_g) * dg + (-w_sg) * dsg);
    }
  }
  double* c = comps + 4 * n;
  c[0] = e_lig;
  c[1] = e_rest;
  c[2] = psi_sg;
  c[3] = psi_g;
}

__global__ void grid_prepare64_kernel(int64_t n, const double* __restrict__ ljr, const double* __restrict__ lja,
                                      const double* __restrict__ elec, double vmax_r, double vmax_e, Hard64* hard,
                                      Soft64* soft) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  double v = ljr[p];
  if (!(v <= kRepulsiveNodeCap)) v = v > 0.0 ? kRepulsiveNodeCap : v;  // caps +inf as well
  if (!(v >= 0.0)) v = 0.0;
  const double e = elec[p];
  hard[p] = Hard64{pow(v, 0.25), lja[p], e, 0.0};
  soft[p] = Soft64{isinf(vmax_r) ? pow(v, 0.25) : pow(vmax_r * tanh(v / vmax_r), 0.25),
                   isinf(vmax_e) ? e : vmax_e * tanh(e / vmax_e)};
}

}  // namespace

cudaError_t launch_grid_prepare64(cudaStream_t s, size_t n_nodes, const double* ljr, const double* lja,
                                  const double* elec, double vmax_r, double vmax_e, Hard64* hard, Soft64* soft) {
  const int threads = 256;
  grid_prepare64_kernel<<<(unsigned)((n_nodes + threads - 1) / threads), threads, 0, s>>>(
      (int64_t)n_nodes, ljr, lja, elec, vmax_r, vmax_e, hard, soft);
  return cudaGetLastError();
}

cudaError_t launch_eval64(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of, const float* x,
                          double* force, double* comps) {
  if (N == 0) return cudaSuccess;
  const int threads = 128;
  eval64_kernel<<<(unsigned)((N + threads - 1) / threads), threads, 0, s>>>(N, c.lig64, c.d_lig64, c.grid64,
                                                                          c.d_states, c.K, state_of, x, force, comps);
  return cudaGetLastError();
}

}  // namespace algdock
