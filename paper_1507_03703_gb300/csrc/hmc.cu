// The fused HMC trial ("Sampling"): momentum draw, n_steps of velocity Verlet over the grid
// interaction energy ("Thermodynamic Cycle"), the ligand force field and the flat-bottom
// restraint (Eq. (binding_site)), then the Metropolis test on the total energy change.
//
// Layout: one warp per replica; lane l owns atoms l, l+32, l+64 (APL = atoms per lane).  Positions,
// velocities and forces of owned atoms stay in registers for the whole trajectory; the current
// positions are mirrored in a per-warp shared-memory array so that every lane can read every atom.
// The ligand's parameters and topology are staged once per CTA in shared memory.
//
// One force evaluation:
//   1. bonded terms, one term per lane: each term's forces on its 2-4 atoms go to per-warp
//      shared-memory slots (role-major, so consecutive lanes write consecutive words);
//   2. per owned atom: the 8-corner gathers of the grid lattices and the sum of its bonded slots
//      in a fixed order;
//   3. nonbonded pairs, each owned atom against every other atom (the pair type table marks
//      excluded and 1-4 pairs); when the last pass has at most 16 atoms, two lanes share an atom
//      and split the partner range;
//   4. the restraint on the warp-reduced centre of mass.
// Every force is accumulated by one lane in a fixed order (no atomics), so results are
// deterministic.
#include <math.h>

#include <algorithm>

#include "internal.cuh"

namespace algdock {
namespace {

constexpr int kWarpsPerBlock = 4;
constexpr unsigned kFull = 0xffffffffu;

struct Lig {
  const float4* atom_a;  // (accel factor 4.184e-4/m, q, sqrt(A), sqrt(B))
  const float4* atom_b;  // (R*, sqrt(eps), m, sqrt(accel factor))
  const uint8_t* ptype;  // [j][i]: 0 nonbonded, 1 1-4, 2 excluded (and i == j)
  const float4* bond;
  const int4* ang_i;
  const float4* ang_p;
  const int4* tor_i;
  const float4* tor_v;
  const float4* tor_c;
  const float4* tor_s;
  const uint2* gs;  // gather schedule: [gs_iters][32] words of four 16-bit entries
  const uint2* gp;  // [na]: four 16-bit partial-sum slots per atom
  const float4* pair;   // [p][i]: records of atom i with partners 2p, 2p + 1 (only where the table is staged)
};

__device__ inline Lig bind_ligand(const uint32_t* s, const LigandLayout& L) {
  Lig g;
  g.atom_a = (const float4*)(s + L.off_atom_a);
  g.atom_b = (const float4*)(s + L.off_atom_b);
  g.ptype = (const uint8_t*)(s + L.off_ptype);
  g.bond = (const float4*)(s + L.off_bond);
  g.ang_i = (const int4*)(s + L.off_ang);
  g.ang_p = (const float4*)(s + L.off_ang + 4 * L.nang);
  g.tor_i = (const int4*)(s + L.off_tor);
  g.tor_v = (const float4*)(s + L.off_tor + 4 * L.ntor);
  g.tor_c = (const float4*)(s + L.off_tor + 8 * L.ntor);
  g.tor_s = (const float4*)(s + L.off_tor + 12 * L.ntor);
  g.gs = (const uint2*)(s + L.off_gs);
  g.gp = (const uint2*)(s + L.off_gp);
  g.pair = (const float4*)(s + L.off_pair);
  return g;
}

__device__ inline double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ inline float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Lattice coordinate of x along one axis.  x - o is formed exactly as s + e (two-sum), so the
// fractional offset keeps FP32 precision relative to the cell even far from the origin.
__device__ inline void axis_coord(float x, float o, float inv_h, int n, int& c, float& t, bool& inside) {
  const float a = x, b = -o;
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  float u = s * inv_h;
  const float ue = e * inv_h;
  inside = true;
  float fl = floorf(u);
  float frac = (u - fl) + ue;
  if (!(u + ue >= 0.f)) {  // below the lattice, or NaN
    fl = 0.f;
    frac = 0.f;
    inside = false;
  } else if (!(fl + frac < (float)(n - 1))) {  // at or beyond the last node, including u = +inf
    fl = (float)(n - 2);
    frac = 1.f;
    if (u + ue > (float)(n - 1)) inside = false;
  } else if (frac >= 1.f) {  // ue pushed the offset into the next cell
    fl += 1.f;
    frac -= 1.f;
  } else if (frac < 0.f) {
    fl -= 1.f;
    frac += 1.f;
  }
  c = (int)fl;
  t = frac;
}

struct GridOut {
  float e_g, e_sg;   // Psi_g, Psi_sg contributions of this atom
  float fx, fy, fz;  // -(w_sg dPsi_sg + w_g dPsi_g)/dx
  bool outside;
};

// Trilinear value and gradient (in lattice units) of two channels at once from the 8 corner values
// c_zyx, in paired FP32 instructions: per channel, the edge differences along x and the values
// interpolated along x, then along y (with the y and x gradients), then along z.  Each half
// performs the operations of the one-channel interpolant in the same order.
struct Tri2 {
  f32x2 v, gx, gy, gz;
};
__device__ inline Tri2 tri2(f32x2 c000, f32x2 c001, f32x2 c010, f32x2 c011, f32x2 c100, f32x2 c101, f32x2 c110,
                            f32x2 c111, f32x2 tx, f32x2 ty, f32x2 tz) {
  const f32x2 d00 = sub2(c001, c000), d01 = sub2(c011, c010), d10 = sub2(c101, c100), d11 = sub2(c111, c110);
  const f32x2 a00 = fma2(tx, d00, c000), a01 = fma2(tx, d01, c010);
  const f32x2 a10 = fma2(tx, d10, c100), a11 = fma2(tx, d11, c110);
  const f32x2 by0 = sub2(a01, a00), by1 = sub2(a11, a10);
  const f32x2 b0 = fma2(ty, by0, a00), b1 = fma2(ty, by1, a10);
  const f32x2 bx0 = fma2(ty, sub2(d01, d00), d00), bx1 = fma2(ty, sub2(d11, d10), d10);
  Tri2 r;
  r.gz = sub2(b1, b0);
  r.v = fma2(tz, r.gz, b0);
  r.gx = fma2(tz, sub2(bx1, bx0), bx0);
  r.gy = fma2(tz, sub2(by1, by0), by0);
  return r;
}
__device__ inline f32x2 lo2(float4 c) { return pack2(c.x, c.y); }
__device__ inline f32x2 hi2(float4 c) { return pack2(c.z, c.w); }

// Grid energies and forces of one atom.  hard / soft select which lattices are read.  The hard
// lattice's channels run as the pairs (LJr^1/4, LJa) and (elec, 0), the soft lattice's as one pair.
__device__ inline GridOut grid_atom(const GridDev& G, float x, float y, float z, float sA, float sB, float q,
                                    bool hard, bool soft, float w_sg, float w_g) {
  GridOut o{0.f, 0.f, 0.f, 0.f, 0.f, false};
  int cx, cy, cz;
  float tx, ty, tz;
  bool ix, iy, iz;
  axis_coord(x, G.ox, G.inv_h, G.nx, cx, tx, ix);
  axis_coord(y, G.oy, G.inv_h, G.ny, cy, ty, iy);
  axis_coord(z, G.oz, G.inv_h, G.nz, cz, tz, iz);
  o.outside = !(ix && iy && iz);
  const float mx = ix ? G.inv_h : 0.f, my = iy ? G.inv_h : 0.f, mz = iz ? G.inv_h : 0.f;
  const int64_t sy = G.nx, sz = (int64_t)G.nx * G.ny;
  const int64_t b = (int64_t)cz * sz + (int64_t)cy * sy + cx;
  const f32x2 tx2 = pack2(tx, tx), ty2 = pack2(ty, ty), tz2 = pack2(tz, tz);
  f32x2 gx2 = 0ull, gy2 = 0ull, gz2 = 0ull;  // (sum of the weighted channel gradients) in two halves
  if (hard) {  // four x-pair records: corners (x, x+1) of each (y, z) edge in one 32-byte load
    float4 c000, c001, c010, c011, c100, c101, c110, c111;
    ldg_pair(G.hard + 2 * b, c000, c001);
    ldg_pair(G.hard + 2 * (b + sy), c010, c011);
    ldg_pair(G.hard + 2 * (b + sz), c100, c101);
    ldg_pair(G.hard + 2 * (b + sz + sy), c110, c111);
    const Tri2 ra = tri2(lo2(c000), lo2(c001), lo2(c010), lo2(c011), lo2(c100), lo2(c101), lo2(c110), lo2(c111), tx2,
                         ty2, tz2);
    const Tri2 e0 = tri2(hi2(c000), hi2(c001), hi2(c010), hi2(c011), hi2(c100), hi2(c101), hi2(c110), hi2(c111), tx2,
                         ty2, tz2);
    float rv, av, ev, zv;
    unpack2(ra.v, rv, av);
    unpack2(e0.v, ev, zv);
    const float r2 = rv * rv;
    o.e_g = sA * (r2 * r2) + sB * av + q * ev;
    if (w_g != 0.f) {
      const float cr = 4.f * sA * r2 * rv;
      const f32x2 kra = pack2(w_g * cr, w_g * sB), ke = pack2(w_g * q, 0.f);
      gx2 = fma2(kra, ra.gx, mul2(ke, e0.gx));
      gy2 = fma2(kra, ra.gy, mul2(ke, e0.gy));
      gz2 = fma2(kra, ra.gz, mul2(ke, e0.gz));
    }
  }
  if (soft) {  // two (x, y) quad records: the corners of the cell's lower and upper z face
    float4 e00, e01, e10, e11;
    ldg_pair(G.soft + 2 * b, e00, e01);
    ldg_pair(G.soft + 2 * (b + sz), e10, e11);
    const Tri2 re = tri2(lo2(e00), hi2(e00), lo2(e01), hi2(e01), lo2(e10), hi2(e10), lo2(e11), hi2(e11), tx2, ty2, tz2);
    float rv, ev;
    unpack2(re.v, rv, ev);
    const float r2 = rv * rv;
    o.e_sg = sA * (r2 * r2) + q * ev;
    if (w_sg != 0.f) {
      const f32x2 k = pack2(w_sg * (4.f * sA * r2 * rv), w_sg * q);
      gx2 = fma2(k, re.gx, gx2);
      gy2 = fma2(k, re.gy, gy2);
      gz2 = fma2(k, re.gz, gz2);
    }
  }
  float ga, gb;
  unpack2(gx2, ga, gb);
  o.fx = -(ga + gb) * mx;
  unpack2(gy2, ga, gb);
  o.fy = -(ga + gb) * my;
  unpack2(gz2, ga, gb);
  o.fz = -(ga + gb) * mz;
  return o;
}

struct Energies {
  float lig;    // bonded + nonbonded (pairs counted from both ends, halved)
  float rest;   // restraint
  float sg, g;  // grid terms
};

__device__ inline float3 sub(float4 a, float4 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ inline float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ inline float3 cross(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ inline void put(float4* sl, int s, float3 f) { sl[s] = make_float4(f.x, f.y, f.z, 0.f); }

// Step 1: every bonded term once, one per lane; per-role forces to the warp's float4 slots.
// Slots: bond t role r -> r*nb + t; angle -> 2nb + r*nang + t; torsion -> 2nb + 3nang + r*ntor + t.
template <bool ENERGY, bool FORCES = true>
__device__ inline float bonded_terms(const Lig& L, const LigandLayout& LL, const float4* xs, float4* sl) {
  const int lane = threadIdx.x & 31;
  float e = 0.f;
  const int nb = LL.nb, nang = LL.nang, ntor = LL.ntor;
  for (int t = lane; t < nb; t += 32) {  // k (r - r0)^2
    const float4 bp = L.bond[t];
    const float3 d = sub(xs[__float_as_int(bp.x)], xs[__float_as_int(bp.y)]);
    const float r2 = dot(d, d);
    const float inv_r = rsqrtf(r2);
    const float dr = r2 * inv_r - bp.w;
    if (ENERGY) e += bp.z * dr * dr;
    const float c = -2.f * bp.z * dr * inv_r;
    if (FORCES) put(sl, t, make_float3(c * d.x, c * d.y, c * d.z));
    if (FORCES) put(sl, nb + t, make_float3(-c * d.x, -c * d.y, -c * d.z));
  }
  const int ab = 2 * nb;
  for (int t = lane; t < nang; t += 32) {  // k (theta - theta0)^2
    const int4 id = L.ang_i[t];
    const float4 ap = L.ang_p[t];
    const float3 u = sub(xs[id.x], xs[id.y]);
    const float3 w = sub(xs[id.z], xs[id.y]);
    const float lu2 = dot(u, u), lw2 = dot(w, w);
    const float inv_luw = rsqrtf(lu2 * lw2);
    const float c = fminf(1.f, fmaxf(-1.f, dot(u, w) * inv_luw));
    const float dth = acosf(c) - ap.y;
    if (ENERGY) e += ap.x * dth * dth;
    const float coef = 2.f * ap.x * dth * rsqrtf(fmaxf(1.f - c * c, 1e-12f));
    const float cu = __fdividef(coef * c, lu2), cw = __fdividef(coef * c, lw2), cx = coef * inv_luw;
    const float3 fa = make_float3(cx * w.x - cu * u.x, cx * w.y - cu * u.y, cx * w.z - cu * u.z);
    const float3 fc = make_float3(cx * u.x - cw * w.x, cx * u.y - cw * w.y, cx * u.z - cw * w.z);
    if (FORCES) put(sl, ab + t, fa);
    if (FORCES) put(sl, ab + nang + t, make_float3(-(fa.x + fc.x), -(fa.y + fc.y), -(fa.z + fc.z)));
    if (FORCES) put(sl, ab + 2 * nang + t, fc);
  }
  const int tb = ab + 3 * nang;
  for (int t = lane; t < ntor; t += 32) {  // sum_n V_n/2 (1 + cos(n phi - gamma_n))
    const int4 id = L.tor_i[t];
    const float4 V = L.tor_v[t], cg = L.tor_c[t], sg = L.tor_s[t];
    const float3 b1 = sub(xs[id.y], xs[id.x]);
    const float3 b2 = sub(xs[id.z], xs[id.y]);
    const float3 b3 = sub(xs[id.w], xs[id.z]);
    const float3 n1 = cross(b1, b2), n2 = cross(b2, b3);
    const float lb22 = dot(b2, b2);
    const float inv_lb2 = rsqrtf(lb22);
    const float lb2 = lb22 * inv_lb2;
    const float n1s = fmaxf(dot(n1, n1), 1e-20f), n2s = fmaxf(dot(n2, n2), 1e-20f);
    const float inv = rsqrtf(n1s * n2s);
    const float cp = dot(n1, n2) * inv;        // cos phi
    const float sp = lb2 * dot(b1, n2) * inv;  // sin phi
    const float c2 = 2.f * cp * cp - 1.f, s2 = 2.f * sp * cp;
    const float c3 = cp * (4.f * cp * cp - 3.f), s3 = sp * (3.f - 4.f * sp * sp);
    if (ENERGY)
      e += V.x * (1.f + cp * cg.x + sp * sg.x) + V.y * (1.f + c2 * cg.y + s2 * sg.y) +
           V.z * (1.f + c3 * cg.z + s3 * sg.z);
    // dE/dphi = sum_n V_n/2 n (cos(n phi) sin g - sin(n phi) cos g)
    const float dE = V.x * (cp * sg.x - sp * cg.x) + 2.f * V.y * (c2 * sg.y - s2 * cg.y) +
                     3.f * V.z * (c3 * sg.z - s3 * cg.z);
    const float ai = __fdividef(dE * lb2, n1s), al = -__fdividef(dE * lb2, n2s);  // F_i = ai n1, F_l = al n2
    const float inv_lb22 = inv_lb2 * inv_lb2;
    const float p = dot(b1, b2) * inv_lb22, q = dot(b3, b2) * inv_lb22;
    const float3 fi = make_float3(ai * n1.x, ai * n1.y, ai * n1.z);
    const float3 fl = make_float3(al * n2.x, al * n2.y, al * n2.z);
    const float3 fj = make_float3(-(1.f + p) * fi.x + q * fl.x, -(1.f + p) * fi.y + q * fl.y,
                                  -(1.f + p) * fi.z + q * fl.z);
    const float3 fk = make_float3(p * fi.x - (1.f + q) * fl.x, p * fi.y - (1.f + q) * fl.y,
                                  p * fi.z - (1.f + q) * fl.z);
    if (FORCES) put(sl, tb + t, fi);
    if (FORCES) put(sl, tb + ntor + t, fj);
    if (FORCES) put(sl, tb + 2 * ntor + t, fk);
    if (FORCES) put(sl, tb + 3 * ntor + t, fl);
  }
  return e;
}

// Step 3: nonbonded pairs.  Pass a covers atoms 32a .. 32a+31; a pass with at most 16 atoms gives
// each atom two lanes, which split the partner range and combine with one shuffle.
template <int APL, bool ENERGY, bool FORCES = true>
__device__ inline void nonbonded(const Lig& L, int na, const float4* xs, float (&F)[APL][3], float& el) {
  const int lane = threadIdx.x & 31;
  float e2 = 0.f;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int base = 32 * a;
    const int m = na - base;
    if (m <= 0) break;
    const bool split = m <= 16;
    const int il = split ? (lane & 15) : lane;
    const int i = base + il;
    const bool act = il < m;
    // partners: all j; split: the low half-warp takes j = 0 .. h-1 upwards, the high half-warp
    // j = na-1 .. h downwards (opposite directions keep the two rows read per step in different
    // shared-memory banks)
    int jb = 0, cnt = na, dir = 1;
    if (split) {
      const int h = (na + 1) >> 1;
      jb = lane < 16 ? 0 : na - 1;
      cnt = lane < 16 ? h : na - h;
      dir = lane < 16 ? 1 : -1;
    }
    float fx = 0.f, fy = 0.f, fz = 0.f;
    if (act) {
      const float4 pi = xs[i];
      const float4 bi = L.atom_b[i];
      const float qi = (float)kCoulomb * pi.w, ri = bi.x, si = bi.y;
      const uint8_t* ty_col = L.ptype + i;
      for (int jj = 0; jj < cnt; ++jj) {
        const int j = jb + dir * jj;
        const float4 pj = xs[j];
        const float2 bj = *(const float2*)&L.atom_b[j];
        const uint32_t ty = ty_col[j * na];
        const bool excluded = ty == 2u;
        const float dx = pi.x - pj.x, dy = pi.y - pj.y, dz = pi.z - pj.z;
        const float r2 = excluded ? 1.f : fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float inv_r = rsqrtf(r2);
        const float inv_r2 = inv_r * inv_r;
        const float R = ri + bj.x;
        const float s2 = R * R * inv_r2;
        const float s6 = s2 * s2 * s2;
        const float eps = excluded ? 0.f : (ty == 1u ? 0.5f : 1.f) * (si * bj.y);
        const float qq = excluded ? 0.f : (ty == 1u ? (float)(1.0 / 1.2) : 1.f) * (qi * pj.w);
        const float eel = qq * inv_r;
        const float fr = fmaf(12.f * eps, s6 * s6 - s6, eel) * inv_r2;
        if (FORCES) {
          fx = fmaf(fr, dx, fx);
          fy = fmaf(fr, dy, fy);
          fz = fmaf(fr, dz, fz);
        }
        if (ENERGY) e2 += fmaf(eps, s6 * s6 - 2.f * s6, eel);
      }
    }
    if (split) {
      fx += __shfl_xor_sync(kFull, fx, 16);
      fy += __shfl_xor_sync(kFull, fy, 16);
      fz += __shfl_xor_sync(kFull, fz, 16);
    }
    if (lane < m && (!split || lane < 16)) {
      F[a][0] += fx;
      F[a][1] += fy;
      F[a][2] += fz;
    }
  }
  if (ENERGY) el += 0.5f * e2;
}

// Step 3 from the pair table: the same passes and lane layout as `nonbonded`, with each pair's
// scaled coefficients read from the table (12 eps_ij s_LJ, 332 q_i q_j s_el; zero for excluded
// pairs and i == j) instead of being formed from per-atom parameters and the pair type.
// R_ij = R*_i + R*_j (Lorentz-Berthelot) is formed in registers.  r^2 is floored at 0.01 A^2 so
// that a zero record meets finite powers (i == j): (R_ij / r)^12 stays below 1e20 for R_ij <= 4 A.
//
// Partners come two at a time (j = 2p, 2p + 1), and the two terms share paired FP32 instructions:
// the positions are read from the pair-interleaved mirror xp (8 floats per partner pair:
// x, x', y, y', z, z', R*, R*'), the coefficients from one 16-byte record per atom and partner
// pair, so that every operand pair arrives in one aligned register pair.  An odd na ends with a
// zero partner (zero position and radius, zero records).  Each half accumulates its own forces and
// energy; the halves are added at the end of a pass.
constexpr float kPairMinR2 = 1.0e-2f;

// Writes atom i's coordinates into the pair-interleaved mirror.
__device__ inline void put_pair_pos(float* xp, int i, float x, float y, float z) {
  float* b = xp + 8 * (i >> 1) + (i & 1);
  b[0] = x;
  b[2] = y;
  b[4] = z;
}

template <int APL, bool ENERGY, bool FORCES = true>
__device__ inline void nonbonded_table(const Lig& L, int na, const float4* xs, const float* xp, float (&F)[APL][3],
                                       float& el) {
  const int lane = threadIdx.x & 31;
  const int P = (na + 1) >> 1;
  const f32x2 one = pack2(1.f, 1.f), two = pack2(2.f, 2.f), twelfth = pack2(1.f / 12.f, 1.f / 12.f);
  f32x2 e2 = 0ull;  // (0.f, 0.f)
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int base = 32 * a;
    const int m = na - base;
    if (m <= 0) break;
    const bool split = m <= 16;
    const int il = split ? (lane & 15) : lane;
    const int i = base + il;
    const bool act = il < m;
    int pb = 0, cnt = P, dir = 1;
    if (split) {
      const int h = (P + 1) >> 1;
      pb = lane < 16 ? 0 : P - 1;
      cnt = lane < 16 ? h : P - h;
      dir = lane < 16 ? 1 : -1;
    }
    f32x2 fx2 = 0ull, fy2 = 0ull, fz2 = 0ull;
    if (act) {
      const float4 own = xs[i];  // (x, y, z, R*_i) in the table path
      const f32x2 X = pack2(own.x, own.x), Y = pack2(own.y, own.y), Z = pack2(own.z, own.z);
      const f32x2 Ri = pack2(own.w, own.w);
      const float4* rec = L.pair + (size_t)pb * na + i;
      const float4* pp = (const float4*)xp + 2 * pb;
      const int rstep = dir * na, pstep = 2 * dir;
#pragma unroll 2
      for (int jj = 0; jj < cnt; ++jj) {
        const float4 q0 = pp[0];  // (x, x', y, y')
        const float4 q1 = pp[1];  // (z, z', R*, R*')
        const float4 t = *rec;    // (e, e', c, c')
        pp += pstep;
        rec += rstep;
        const f32x2 dx = sub2(X, pack2(q0.x, q0.y)), dy = sub2(Y, pack2(q0.z, q0.w));
        const f32x2 dz = sub2(Z, pack2(q1.x, q1.y));
        float ra, rb;
        unpack2(fma2(dx, dx, fma2(dy, dy, mul2(dz, dz))), ra, rb);
        const f32x2 inv_r = pack2(rsqrtf(fmaxf(ra, kPairMinR2)), rsqrtf(fmaxf(rb, kPairMinR2)));
        const f32x2 R = add2(Ri, pack2(q1.z, q1.w));
        const f32x2 inv_r2 = mul2(inv_r, inv_r);
        const f32x2 s2 = mul2(mul2(R, R), inv_r2);
        const f32x2 s6 = mul2(mul2(s2, s2), s2);
        const f32x2 e = pack2(t.x, t.y);
        const f32x2 eel = mul2(pack2(t.z, t.w), inv_r);
        if (FORCES) {
          const f32x2 fr = mul2(fma2(e, mul2(s6, sub2(s6, one)), eel), inv_r2);
          fx2 = fma2(fr, dx, fx2);
          fy2 = fma2(fr, dy, fy2);
          fz2 = fma2(fr, dz, fz2);
        }
        if (ENERGY) e2 = add2(e2, fma2(mul2(e, twelfth), mul2(s6, sub2(s6, two)), eel));
      }
    }
    float fx, fy, fz, ha, hb;
    unpack2(fx2, fx, ha);
    fx += ha;
    unpack2(fy2, fy, ha);
    fy += ha;
    unpack2(fz2, fz, hb);
    fz += hb;
    if (split) {
      fx += __shfl_xor_sync(kFull, fx, 16);
      fy += __shfl_xor_sync(kFull, fy, 16);
      fz += __shfl_xor_sync(kFull, fz, 16);
    }
    if (lane < m && (!split || lane < 16)) {
      F[a][0] += fx;
      F[a][1] += fy;
      F[a][2] += fz;
    }
  }
  if (ENERGY) {
    float ea, eb;
    unpack2(e2, ea, eb);
    el += 0.5f * (ea + eb);
  }
}

// Step 2a: the bonded forces gathered over the lanes' balanced runs of the atom-sorted slot list
// (the gather schedule): each lane adds its run in order and stores the partial sum of every atom
// it ends in that atom's last slot of the run.
__device__ inline void gather_runs(const Lig& L, const LigandLayout& LL, float4* sl) {
  const int lane = threadIdx.x & 31;
  float ax = 0.f, ay = 0.f, az = 0.f;
  const uint2* gs = L.gs + lane;
  for (int j = 0; j < LL.gs_iters; ++j) {
    const uint2 w = gs[32 * j];
    const uint32_t e[4] = {w.x & 0xffffu, w.x >> 16, w.y & 0xffffu, w.y >> 16};
    float4 v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = sl[e[k] & 0x7fffu];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      ax += v[k].x;
      ay += v[k].y;
      az += v[k].z;
      if (e[k] & 0x8000u) {
        sl[e[k] & 0x7fffu] = make_float4(ax, ay, az, 0.f);
        ax = ay = az = 0.f;
      }
    }
  }
}

// Forces on the lane's atoms (and, if ENERGY, the lane's partial energies).  xs holds all
// positions (x, y, z, q), with R*_i in place of q when TABLE; sl is the warp's bonded-slot scratch
// (n_slots + 1 float4, the last zero).
template <int APL, bool ENERGY, bool TABLE = false, bool FORCES = true>
__device__ inline void evaluate(const LigandLayout& LL, const Lig& L, const GridDev& G, const float4* xs, float4* sl,
                                const float (&x)[APL][3], const float (&mass)[APL], float (&F)[APL][3], float w_sg,
                                float w_g, bool all_grids, Energies& en, int& outside, const float* xp = nullptr) {
  const int lane = threadIdx.x & 31;
  const int na = LL.na;
  float el = bonded_terms<ENERGY, FORCES>(L, LL, xs, sl);
  __syncwarp();
  if (FORCES) {
    gather_runs(L, LL, sl);
    __syncwarp();
  }
  const bool hard = all_grids || w_g != 0.f;
  const bool soft = all_grids || w_sg != 0.f;
  float eg = 0.f, esg = 0.f;
  float mx = 0.f, my = 0.f, mz = 0.f;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    F[a][0] = F[a][1] = F[a][2] = 0.f;
    if (i >= na) continue;
    const float4 pa = L.atom_a[i];
    mx += mass[a] * x[a][0];
    my += mass[a] * x[a][1];
    mz += mass[a] * x[a][2];
    if (hard || soft) {
      const GridOut go = grid_atom(G, x[a][0], x[a][1], x[a][2], pa.z, pa.w, pa.y, hard, soft, FORCES ? w_sg : 0.f,
                                   FORCES ? w_g : 0.f);
      F[a][0] += go.fx;
      F[a][1] += go.fy;
      F[a][2] += go.fz;
      eg += go.e_g;
      esg += go.e_sg;
      outside += go.outside ? 1 : 0;
    }
    if (FORCES) {  // the atom's partial sums, in run order
      const uint2 p = L.gp[i];
      const float4 q0 = sl[p.x & 0xffffu], q1 = sl[p.x >> 16], q2 = sl[p.y & 0xffffu], q3 = sl[p.y >> 16];
      F[a][0] += ((q0.x + q1.x) + q2.x) + q3.x;
      F[a][1] += ((q0.y + q1.y) + q2.y) + q3.y;
      F[a][2] += ((q0.z + q1.z) + q2.z) + q3.z;
    }
  }
  if (TABLE) nonbonded_table<APL, ENERGY, FORCES>(L, na, xs, xp, F, el);
  else nonbonded<APL, ENERGY, FORCES>(L, na, xs, F, el);
  // restraint on the centre of mass
  mx = warp_sumf(mx);
  my = warp_sumf(my);
  mz = warp_sumf(mz);
  const float invM = 1.f / LL.total_mass;
  const float dx = mx * invM - LL.site[0], dy = my * invM - LL.site[1], dz = mz * invM - LL.site[2];
  const float d = sqrtf(dx * dx + dy * dy + dz * dz);
  float er = 0.f;
  if (d > LL.d0) {
    const float ex = d - LL.d0;
    er = 0.5f * LL.k_rest * ex * ex;
    const float c = -LL.k_rest * ex / d * invM;
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i >= na) continue;
      F[a][0] += c * mass[a] * dx;
      F[a][1] += c * mass[a] * dy;
      F[a][2] += c * mass[a] * dz;
    }
  } else if (!(d <= LL.d0)) {  // NaN centre of mass: make the energy NaN
    er = d;
  }
  en.lig = el;
  en.rest = lane == 0 ? er : 0.f;
  en.sg = esg;
  en.g = eg;
}

__device__ inline void reduce_components(const Energies& e, double c[4]) {
  c[0] = warp_sum((double)e.lig);
  c[1] = warp_sum((double)e.rest);
  c[2] = warp_sum((double)e.sg);
  c[3] = warp_sum((double)e.g);
}

// U_k = ((U_L + U_I) + w_sg Psi_sg) + w_g Psi_g, a zero weight dropping its term.
__device__ inline double weighted(const double c[4], double w_sg, double w_g) {
  double e = __dadd_rn(c[0], c[1]);
  if (w_sg != 0.0) e = __dadd_rn(e, __dmul_rn(w_sg, c[2]));
  if (w_g != 0.0) e = __dadd_rn(e, __dmul_rn(w_g, c[3]));
  return e;
}

__device__ inline void stage_ligand(uint32_t* s, const uint32_t* __restrict__ blob, int words) {
  const uint4* src = (const uint4*)blob;
  uint4* dst = (uint4*)s;
  for (int i = threadIdx.x; i < words / 4; i += blockDim.x) dst[i] = src[i];
}

// Shared memory of one block: ligand blob, then per warp 32*APL float4 positions, with the pair
// table also the pair-interleaved mirror of the pair loop (32*APL * 4 floats), and the bonded-slot
// scratch (n_slots + 1 float4, the last a zero slot).
__host__ __device__ inline int scratch_words(const LigandLayout& L) { return 4 * (L.n_slots + 1); }
__host__ __device__ inline int warp_words(const LigandLayout& L, int apl, bool table) {
  return (table ? 8 : 4) * 32 * apl + scratch_words(L);
}

struct WarpSmem {
  float4* xs;
  float* xp;  // pair-interleaved positions (table kernels only)
  float4* sl;  // bonded-force slots
};
template <int APL, bool TABLE = false>
__device__ inline WarpSmem warp_smem(uint32_t* smem, int staged_words, const LigandLayout& LL, int warp) {
  uint32_t* p = smem + staged_words + warp * warp_words(LL, APL, TABLE);
  float* xp = TABLE ? (float*)(p + 4 * 32 * APL) : nullptr;
  float4* sl = (float4*)(p + (TABLE ? 8 : 4) * 32 * APL);
  if ((threadIdx.x & 31) == 0) sl[LL.n_slots] = make_float4(0.f, 0.f, 0.f, 0.f);  // the zero slot
  return WarpSmem{(float4*)p, xp, sl};
}

struct HmcArgs {
  GridDev G;
  LigandLayout LL;
  const uint32_t* blob;
  const StateDev* states;
  int n_states;
  int64_t n_rep;
  const int32_t* state_of;
  float* x;
  double* comps;
  double* dH;
  uint8_t* acc;
  int n_steps;
  uint64_t seed;
  uint32_t cycle;
  int64_t rep_offset;
  int64_t* counters;
  // batches only: the ligand records, this launch's work items (one per block) and the position
  // stride of a replica (atoms)
  const BatchLigand* bligs;
  const BatchItem* items;
  int x_stride;
  unsigned long long* work;  // single-ligand launches: replicas handed out so far (zero at launch), or NULL
};

// One HMC trial of replica r by the calling warp: momenta, n_steps of velocity Verlet, the
// Metropolis test, and the write-back of an accepted trial.  xs / xp / sl are the warp's
// shared-memory arrays (the zero partner of an odd atom count is already in xp).
template <int APL, bool TABLE, bool BATCH>
__device__ __forceinline__ void hmc_trial(const HmcArgs& A, const LigandLayout& LL, const Lig& L, const WarpSmem& ws,
                                          int64_t r) {
  const int lane = threadIdx.x & 31;
  float4* xs = ws.xs;
  float* xp = ws.xp;
  const int na = LL.na;
  const int64_t xstride = BATCH ? A.x_stride : na;
  const int k = A.state_of[r];
  if ((unsigned)k >= (unsigned)A.n_states) {  // invalid state index: leave the replica untouched
    if (lane == 0) {
      if (A.dH) A.dH[r] = __longlong_as_double(0x7ff8000000000000ll);
      if (A.acc) A.acc[r] = 0;
    }
    return;
  }
  const StateDev st = A.states[k];
  const float dt = st.dt, hdt = 0.5f * st.dt;
  const uint32_t rid = (uint32_t)(A.rep_offset + r);

  float x[APL][3], v[APL][3], F[APL][3];
  float mass[APL], accel[APL];  // the lane's atoms' masses and force-to-acceleration factors
  float kin = 0.f;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na) {
      const float* src = A.x + (r * xstride + i) * 3;
      x[a][0] = src[0];
      x[a][1] = src[1];
      x[a][2] = src[2];
      const U4 o = philox(A.seed, (uint32_t)i, rid, A.cycle, kPurposeMomentum);
      // Box-Muller: u1 in (0, 1] from 23 bits + 1/2, u2 in [0, 1) from 23 bits (exact in FP32)
      const float u1 = ((float)(o.x >> 9) + 0.5f) * (1.0f / 8388608.0f);
      const float u2 = (float)(o.y >> 9) * (1.0f / 8388608.0f);
      const float u3 = ((float)(o.z >> 9) + 0.5f) * (1.0f / 8388608.0f);
      const float u4 = (float)(o.w >> 9) * (1.0f / 8388608.0f);
      const float rr1 = sqrtf(-2.f * logf(u1)), rr2 = sqrtf(-2.f * logf(u3));
      float s1, c1, s2, c2;
      sincospif(2.f * u2, &s1, &c1);
      sincospif(2.f * u4, &s2, &c2);
      const float4 pb = L.atom_b[i];
      mass[a] = pb.z;
      accel[a] = L.atom_a[i].x;
      const float sd = st.sqrt_kT * pb.w;  // sqrt(kT * 4.184e-4 / m)
      v[a][0] = rr1 * c1 * sd;
      v[a][1] = rr1 * s1 * sd;
      v[a][2] = rr2 * c2 * sd;
      kin += pb.z * (v[a][0] * v[a][0] + v[a][1] * v[a][1] + v[a][2] * v[a][2]);
      // the fourth component: the charge for the pair-type loop, R*_i for the table loop (which
      // reads the partners' positions and radii from the pair-interleaved mirror)
      xs[i] = make_float4(x[a][0], x[a][1], x[a][2], TABLE ? pb.x : L.atom_a[i].y);
      if (TABLE) {
        put_pair_pos(xp, i, x[a][0], x[a][1], x[a][2]);
        xp[8 * (i >> 1) + 6 + (i & 1)] = pb.x;  // R*_i
      }
    } else {
      x[a][0] = x[a][1] = x[a][2] = 0.f;
      v[a][0] = v[a][1] = v[a][2] = 0.f;
      mass[a] = accel[a] = 0.f;
    }
  }
  __syncwarp();
  int outside = 0;
  Energies en;
  double c[4];
  evaluate<APL, true, TABLE>(LL, L, A.G, xs, ws.sl, x, mass, F, st.w_sg_f, st.w_g_f, true, en, outside, xp);
  reduce_components(en, c);
  // the starting components go out now (a rejected trial leaves them); only U0 stays live
  const double U0 = weighted(c, st.w_sg, st.w_g);
  if (lane < 4) A.comps[r * 4 + lane] = lane == 0 ? c[0] : (lane == 1 ? c[1] : (lane == 2 ? c[2] : c[3]));
  double U1 = U0;
  const double K0 = 0.5 * kKineticToKcal * warp_sum((double)kin);
  for (int s = 0; s < A.n_steps; ++s) {
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          v[a][d] = fmaf(hdt * accel[a], F[a][d], v[a][d]);
          x[a][d] = fmaf(dt, v[a][d], x[a][d]);
        }
      }
    }
    __syncwarp();  // all lanes finished reading the previous positions and bonded slots
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na) {
        float4 p = xs[i];
        p.x = x[a][0];
        p.y = x[a][1];
        p.z = x[a][2];
        xs[i] = p;
        if (TABLE) put_pair_pos(xp, i, x[a][0], x[a][1], x[a][2]);
      }
    }
    __syncwarp();
    if (s + 1 < A.n_steps) {
      evaluate<APL, false, TABLE>(LL, L, A.G, xs, ws.sl, x, mass, F, st.w_sg_f, st.w_g_f, false, en, outside, xp);
    } else {
      evaluate<APL, true, TABLE>(LL, L, A.G, xs, ws.sl, x, mass, F, st.w_sg_f, st.w_g_f, true, en, outside, xp);
      reduce_components(en, c);
      U1 = weighted(c, st.w_sg, st.w_g);
    }
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na) {
#pragma unroll
        for (int d = 0; d < 3; ++d) v[a][d] = fmaf(hdt * accel[a], F[a][d], v[a][d]);
      }
    }
  }
  kin = 0.f;
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na) kin += mass[a] * (v[a][0] * v[a][0] + v[a][1] * v[a][1] + v[a][2] * v[a][2]);
  }
  const double K1 = 0.5 * kKineticToKcal * warp_sum((double)kin);
  const double dH = (K1 + U1) - (K0 + U0);
  const U4 o = philox(A.seed, 0u, rid, A.cycle, kPurposeAccept);
  const double u = uniform53(o.x, o.y);
  const bool accept = u < exp(-dH / st.kT);
  if (accept) {  // a rejected trial leaves the stored positions and components as they were
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na) {
        float* dst = A.x + (r * xstride + i) * 3;
        dst[0] = x[a][0];
        dst[1] = x[a][1];
        dst[2] = x[a][2];
      }
    }
    if (A.n_steps > 0 && lane < 4)
      A.comps[r * 4 + lane] = lane == 0 ? c[0] : (lane == 1 ? c[1] : (lane == 2 ? c[2] : c[3]));
  }
  if (lane == 0) {
    if (A.dH) A.dH[r] = dH;
    if (A.acc) A.acc[r] = accept ? 1 : 0;
  }
  if (A.counters) {
    const int out_total = __reduce_add_sync(kFull, outside);
    if (lane == 0) {
      if (accept) atomicAdd((unsigned long long*)&A.counters[ALGDOCK_CNT_ACCEPTED], 1ull);
      if (!isfinite(dH)) atomicAdd((unsigned long long*)&A.counters[ALGDOCK_CNT_NONFINITE], 1ull);
      if (out_total) atomicAdd((unsigned long long*)&A.counters[ALGDOCK_CNT_OUTSIDE], (unsigned long long)out_total);
    }
  }
}


// WPB warps per block; TABLE: the pair table is staged with the blob (16-warp blocks share it).
// BATCH: the block's ligand and replicas come from its work item (a run of up to WPB replicas of
// one ligand of a multi-ligand batch) and positions are stored x_stride atoms apart.
// Otherwise, with A.work set, the blocks are persistent: each warp takes replicas from the work
// counter until all n_rep are handed out, highest index first (the coupling leg, whose trials
// gather the lattices, before the cheaper warming leg), so that no SM idles while another still
// runs a last wave of blocks.  Which warp runs a replica does not change its result.
template <int APL, int WPB, bool TABLE, bool BATCH = false>
__global__ void __launch_bounds__(WPB * 32) hmc_kernel(const HmcArgs A) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ LigandLayout s_ll;
  const uint32_t* blob = A.blob;
  int64_t r_first = (int64_t)blockIdx.x * WPB;
  int count = WPB;
  if (BATCH) {
    const BatchItem it = A.items[blockIdx.x];
    if (threadIdx.x == 0) s_ll = A.bligs[it.lig].LL;
    blob = A.blob + A.bligs[it.lig].blob_off;
    r_first = it.r0;
    count = it.count;
    __syncthreads();
  }
  const LigandLayout& LL = BATCH ? s_ll : A.LL;
  const int staged = TABLE ? LL.words_pair : LL.words;
  stage_ligand(smem, blob, staged);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= count) return;
  const Lig L = bind_ligand(smem, LL);
  const WarpSmem ws = warp_smem<APL, TABLE>(smem, staged, LL, warp);
  const int na = LL.na;
  if (TABLE && (na & 1) && lane == 0) {  // the zero partner that completes the last pair
    put_pair_pos(ws.xp, na, 0.f, 0.f, 0.f);
    ws.xp[8 * (na >> 1) + 7] = 0.f;
  }
  if (!BATCH && A.work) {
    for (;;) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(A.work, 1ull);
      t = __shfl_sync(kFull, t, 0);
      if (t >= (unsigned long long)A.n_rep) break;
      __syncwarp();  // the previous trial's reads of the warp's shared arrays are done
      hmc_trial<APL, TABLE, BATCH>(A, LL, L, ws, A.n_rep - 1 - (int64_t)t);
    }
    return;
  }
  const int64_t r = r_first + warp;
  if (r >= A.n_rep) return;
  hmc_trial<APL, TABLE, BATCH>(A, LL, L, ws, r);
}

// Energy (and, with force != NULL, force) of stored configurations, one warp each.  With
// state_of == NULL the grid weights are zero (components only).
struct EvalArgs {
  GridDev G;
  LigandLayout LL;
  const uint32_t* blob;
  const StateDev* states;
  int n_states;
  int64_t N;
  const int32_t* state_of;
  const float* x;
  float* force;
  double* comps;
};

// FORCES = false: energies only (the bonded force slots, grid gradients and pair forces are skipped).
template <int APL, bool FORCES>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) eval_kernel(const EvalArgs A) {
  extern __shared__ __align__(16) uint32_t smem[];
  stage_ligand(smem, A.blob, A.LL.words);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (n >= A.N) return;
  const Lig L = bind_ligand(smem, A.LL);
  const WarpSmem ws = warp_smem<APL>(smem, A.LL.words, A.LL, warp);
  const int na = A.LL.na;
  float w_sg = 0.f, w_g = 0.f;
  if (A.state_of) {
    const int k = A.state_of[n];
    if ((unsigned)k >= (unsigned)A.n_states) return;  // invalid state index: no output
    w_sg = A.states[k].w_sg_f;
    w_g = A.states[k].w_g_f;
  }
  float x[APL][3], F[APL][3], mass[APL];
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na) {
      const float* src = A.x + (n * na + i) * 3;
      x[a][0] = src[0];
      x[a][1] = src[1];
      x[a][2] = src[2];
      mass[a] = L.atom_b[i].z;
      ws.xs[i] = make_float4(x[a][0], x[a][1], x[a][2], L.atom_a[i].y);
    } else {
      x[a][0] = x[a][1] = x[a][2] = mass[a] = 0.f;
    }
  }
  __syncwarp();
  Energies en;
  int outside = 0;
  evaluate<APL, true, false, FORCES>(A.LL, L, A.G, ws.xs, ws.sl, x, mass, F, w_sg, w_g, true, en, outside);
  double c[4];
  reduce_components(en, c);
  if (FORCES && A.force) {
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const int i = lane + 32 * a;
      if (i < na) {
        float* dst = A.force + (n * na + i) * 3;
        dst[0] = F[a][0];
        dst[1] = F[a][1];
        dst[2] = F[a][2];
      }
    }
  }
  if (A.comps && lane < 4) A.comps[n * 4 + lane] = c[lane];
}

// External-coordinate moves ("Sampling"): for a replica whose state has alpha < alpha_max, n_moves
// moves, each a uniformly random rotation about the centre of mass (the unit quaternion of three
// uniforms by Shoemake's construction) and a Gaussian translation of sigma per dimension, accepted
// by the Metropolis test on the state's energy.  One warp per replica.  A rigid move leaves the
// intramolecular energy unchanged, so U_L is carried over and only the grid terms and the
// restraint of the moved pose are evaluated (both lattices, so all four components stay current).
// Philox counter {d, replica, cycle * n_moves + move, 5}: d = 0 the quaternion's uniforms, d = 1
// the translation (Box-Muller), d = 2 the accept uniform.
struct ExtArgs {
  GridDev G;
  LigandLayout LL;
  const uint32_t* blob;  // the ligand blob in global memory (read through the cache)
  const StateDev* states;
  int n_states;
  int64_t n_rep;
  const int32_t* state_of;
  float* x;
  double* comps;
  int n_moves;
  double alpha_max;
  float sigma;
  uint64_t seed;
  uint64_t cycle;
  int64_t rep_offset;
  int32_t* accepted;
  int64_t* counters;
};

template <int APL>
__global__ void __launch_bounds__(kWarpsPerBlock * 32) external_kernel(const ExtArgs A) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (r >= A.n_rep) return;
  const int k = A.state_of[r];
  if ((unsigned)k >= (unsigned)A.n_states) return;
  const StateDev st = A.states[k];
  if (!(st.alpha < A.alpha_max)) return;  // also the warming leg's NaN
  const Lig L = bind_ligand(A.blob, A.LL);
  const int na = A.LL.na;
  const uint32_t rid = (uint32_t)(A.rep_offset + r);
  float x[APL][3], sA[APL], sB[APL], q[APL], m[APL];
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    const bool own = i < na;
    const float4 pa = own ? L.atom_a[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    m[a] = own ? L.atom_b[i].z : 0.f;
    q[a] = pa.y;
    sA[a] = pa.z;
    sB[a] = pa.w;
#pragma unroll
    for (int d = 0; d < 3; ++d) x[a][d] = own ? A.x[(r * na + i) * 3 + d] : 0.f;
  }
  double c0[4];
  {
    const double mine = lane < 4 ? A.comps[r * 4 + lane] : 0.0;
#pragma unroll
    for (int c = 0; c < 4; ++c) c0[c] = __shfl_sync(kFull, mine, c);
  }
  const float invM = 1.f / A.LL.total_mass;
  const double u0 = weighted(c0, st.w_sg, st.w_g);
  int n_acc = 0, outside = 0;
  double u_cur = u0;
  for (int mv = 0; mv < A.n_moves; ++mv) {
    const uint32_t ctr = (uint32_t)(A.cycle * (uint64_t)A.n_moves + (uint64_t)mv);
    // rotation
    const U4 rq = philox(A.seed, 0u, rid, ctr, kPurposeExternal);
    const float u1 = (float)(rq.x >> 9) * (1.0f / 8388608.0f);
    const float u2 = (float)(rq.y >> 9) * (1.0f / 8388608.0f);
    const float u3 = (float)(rq.z >> 9) * (1.0f / 8388608.0f);
    const float s1 = sqrtf(1.f - u1), s2 = sqrtf(u1);
    float sn2, cs2, sn3, cs3;
    sincospif(2.f * u2, &sn2, &cs2);
    sincospif(2.f * u3, &sn3, &cs3);
    const float qx = s1 * sn2, qy = s1 * cs2, qz = s2 * sn3, qw = s2 * cs3;
    const float R00 = 1.f - 2.f * (qy * qy + qz * qz), R01 = 2.f * (qx * qy - qz * qw), R02 = 2.f * (qx * qz + qy * qw);
    const float R10 = 2.f * (qx * qy + qz * qw), R11 = 1.f - 2.f * (qx * qx + qz * qz), R12 = 2.f * (qy * qz - qx * qw);
    const float R20 = 2.f * (qx * qz - qy * qw), R21 = 2.f * (qy * qz + qx * qw), R22 = 1.f - 2.f * (qx * qx + qy * qy);
    // translation: Box-Muller on 23-bit uniforms, as for the momenta
    const U4 rt = philox(A.seed, 1u, rid, ctr, kPurposeExternal);
    const float ua = ((float)(rt.x >> 9) + 0.5f) * (1.0f / 8388608.0f), ub = (float)(rt.y >> 9) * (1.0f / 8388608.0f);
    const float uc = ((float)(rt.z >> 9) + 0.5f) * (1.0f / 8388608.0f), ud = (float)(rt.w >> 9) * (1.0f / 8388608.0f);
    float sb, cb, sd_, cd;
    sincospif(2.f * ub, &sb, &cb);
    sincospif(2.f * ud, &sd_, &cd);
    const float ra = sqrtf(-2.f * logf(ua)), rc = sqrtf(-2.f * logf(uc));
    const float tx = A.sigma * ra * cb, ty = A.sigma * ra * sb, tz = A.sigma * rc * cd;
    // centre of mass, moved pose, its grid terms and restraint
    float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      cx += m[a] * x[a][0];
      cy += m[a] * x[a][1];
      cz += m[a] * x[a][2];
    }
    cx = warp_sumf(cx) * invM;
    cy = warp_sumf(cy) * invM;
    cz = warp_sumf(cz) * invM;
    float y[APL][3];
    float eg = 0.f, esg = 0.f, mx = 0.f, my = 0.f, mz = 0.f;
    int out_mv = 0;
#pragma unroll
    for (int a = 0; a < APL; ++a) {
      const float vx = x[a][0] - cx, vy = x[a][1] - cy, vz = x[a][2] - cz;
      y[a][0] = cx + (R00 * vx + R01 * vy + R02 * vz) + tx;
      y[a][1] = cy + (R10 * vx + R11 * vy + R12 * vz) + ty;
      y[a][2] = cz + (R20 * vx + R21 * vy + R22 * vz) + tz;
      if (lane + 32 * a < na) {
        const GridOut go = grid_atom(A.G, y[a][0], y[a][1], y[a][2], sA[a], sB[a], q[a], true, true, 0.f, 0.f);
        eg += go.e_g;
        esg += go.e_sg;
        out_mv += go.outside ? 1 : 0;
        mx += m[a] * y[a][0];
        my += m[a] * y[a][1];
        mz += m[a] * y[a][2];
      }
    }
    mx = warp_sumf(mx);
    my = warp_sumf(my);
    mz = warp_sumf(mz);
    const float dx = mx * invM - A.LL.site[0], dy = my * invM - A.LL.site[1], dz = mz * invM - A.LL.site[2];
    const float d = sqrtf(dx * dx + dy * dy + dz * dz);
    float er = 0.f;
    if (d > A.LL.d0) {
      const float ex = d - A.LL.d0;
      er = 0.5f * A.LL.k_rest * ex * ex;
    } else if (!(d <= A.LL.d0)) {
      er = d;
    }
    double c1[4];
    c1[0] = c0[0];
    c1[1] = (double)er;
    c1[2] = warp_sum((double)esg);
    c1[3] = warp_sum((double)eg);
    const double u1e = weighted(c1, st.w_sg, st.w_g);
    const U4 ra4 = philox(A.seed, 2u, rid, ctr, kPurposeExternal);
    const bool acc = uniform53(ra4.x, ra4.y) < exp(-st.beta * (u1e - u_cur));
    outside += out_mv;
    if (acc) {
#pragma unroll
      for (int a = 0; a < APL; ++a)
#pragma unroll
        for (int dd = 0; dd < 3; ++dd) x[a][dd] = y[a][dd];
#pragma unroll
      for (int c = 0; c < 4; ++c) c0[c] = c1[c];
      u_cur = u1e;
      ++n_acc;
    }
  }
#pragma unroll
  for (int a = 0; a < APL; ++a) {
    const int i = lane + 32 * a;
    if (i < na)
#pragma unroll
      for (int d = 0; d < 3; ++d) A.x[(r * na + i) * 3 + d] = x[a][d];
  }
  if (lane < 4) A.comps[r * 4 + lane] = lane == 0 ? c0[0] : (lane == 1 ? c0[1] : (lane == 2 ? c0[2] : c0[3]));
  if (lane == 0) {
    if (A.accepted) A.accepted[r] += n_acc;
    if (A.counters) {
      if (n_acc) atomicAdd((unsigned long long*)&A.counters[ALGDOCK_CNT_ACCEPTED], (unsigned long long)n_acc);
    }
  }
  if (A.counters) {
    const int out_total = __reduce_add_sync(kFull, outside);
    if (lane == 0 && out_total)
      atomicAdd((unsigned long long*)&A.counters[ALGDOCK_CNT_OUTSIDE], (unsigned long long)out_total);
  }
}

// u_kn[k][n] from stored components (k over k_count states from k_begin).
__global__ void ukn_kernel(const StateDev* __restrict__ states, int k_begin, int k_count, int64_t N,
                           const double* __restrict__ comps, double* u_kn) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  double c[4];
  const double2 c01 = *(const double2*)(comps + 4 * n), c23 = *(const double2*)(comps + 4 * n + 2);
  c[0] = c01.x;
  c[1] = c01.y;
  c[2] = c23.x;
  c[3] = c23.y;
  for (int k = blockIdx.y; k < k_count; k += gridDim.y) {
    const StateDev st = states[k_begin + k];
    u_kn[(int64_t)k * N + n] = __dmul_rn(st.beta, weighted(c, st.w_sg, st.w_g));
  }
}

int atoms_per_lane(int na) { return na <= 32 ? 1 : (na <= 64 ? 2 : 3); }

size_t block_smem(const LigandLayout& L, int apl, int wpb = kWarpsPerBlock, bool table = false) {
  return ((size_t)(table ? L.words_pair : L.words) + (size_t)wpb * warp_words(L, apl, table)) * 4;
}

constexpr int kTableWarps = 16;  // warps per block of the pair-table HMC kernel (512 threads, 128 registers)
constexpr size_t kMaxBlockSmem = 227 * 1024;

template <typename Kernel, typename Args>
cudaError_t launch_templated(Kernel k1, Kernel k2, Kernel k3, int apl, size_t smem, int64_t items, cudaStream_t s,
                             const Args& A, int wpb = kWarpsPerBlock) {
  Kernel k = apl == 1 ? k1 : (apl == 2 ? k2 : k3);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = (items + wpb - 1) / wpb;
  k<<<(unsigned)blocks, wpb * 32, smem, s>>>(A);
  return cudaGetLastError();
}

}  // namespace

bool hmc_uses_table(const LigandLayout& L) {
  const int apl = atoms_per_lane(L.na);
  return apl <= 2 && block_smem(L, apl, kTableWarps, true) <= kMaxBlockSmem;
}

cudaError_t launch_hmc(cudaStream_t s, const algdock_ctx& c, int64_t n_rep, const int32_t* state_of, float* x,
                       double* comps, double* dH, uint8_t* acc, int n_steps, uint64_t seed, uint64_t cycle,
                       int64_t rep_offset, int64_t* counters) {
  if (n_rep == 0) return cudaSuccess;
  HmcArgs A{c.grid, c.lig, c.d_blob, c.d_states, c.K, n_rep, state_of, x, comps, dH, acc, n_steps, seed,
            (uint32_t)cycle, rep_offset, counters, nullptr, nullptr, 0, c.d_work};
  const int apl = atoms_per_lane(c.lig.na);
  // the pair table where 16-warp blocks can stage it (up to 64 atoms with a small topology);
  // otherwise the pair-type path in 4-warp blocks
  const bool table = hmc_uses_table(c.lig);
  void (*k)(const HmcArgs);
  if (table) k = apl == 1 ? hmc_kernel<1, kTableWarps, true> : hmc_kernel<2, kTableWarps, true>;
  else k = apl == 1 ? hmc_kernel<1, kWarpsPerBlock, false>
                    : (apl == 2 ? hmc_kernel<2, kWarpsPerBlock, false> : hmc_kernel<3, kWarpsPerBlock, false>);
  const int wpb = table ? kTableWarps : kWarpsPerBlock;
  const size_t smem = table ? block_smem(c.lig, apl, kTableWarps, true) : block_smem(c.lig, apl);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // persistent blocks: as many as fit on the device at once, never more than the replicas need
  int per_sm = 0, sms = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, wpb * 32, smem);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c.device);
  if (e != cudaSuccess) return e;
  const int64_t need = (n_rep + wpb - 1) / wpb;
  const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)std::max(per_sm, 1) * sms));
  e = cudaMemsetAsync(c.d_work, 0, sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  k<<<(unsigned)blocks, wpb * 32, smem, s>>>(A);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ multi-ligand batches
size_t batch_block_smem(const LigandLayout& L, int apl, int wpb, bool table) { return block_smem(L, apl, wpb, table); }

// Launch shapes tried for a class: pair-table blocks of 16 or 8 replicas, or 4-replica blocks
// without the table (classes 0 and 1); 8-replica table blocks or 4 without (2); 4 or 8 replicas
// without the table (3).
int batch_candidates(int cls, int* wpb, bool* table) {
  if (cls == 3) {
    wpb[0] = 4, table[0] = false;
    wpb[1] = 8, table[1] = false;
    return 2;
  }
  if (cls == 2) {
    wpb[0] = 8, table[0] = true;
    wpb[1] = kWarpsPerBlock, table[1] = false;
    return 2;
  }
  wpb[0] = kTableWarps, table[0] = true;
  wpb[1] = 8, table[1] = true;
  wpb[2] = kWarpsPerBlock, table[2] = false;
  return 3;
}

namespace {
using HmcKernel = void (*)(const HmcArgs);
HmcKernel batch_kernel(int apl, int wpb, bool table) {
  if (apl == 1) {
    if (table) return wpb == kTableWarps ? hmc_kernel<1, kTableWarps, true, true> : hmc_kernel<1, 8, true, true>;
    return hmc_kernel<1, kWarpsPerBlock, false, true>;
  }
  if (apl == 2) {
    if (table) return wpb == kTableWarps ? hmc_kernel<2, kTableWarps, true, true> : hmc_kernel<2, 8, true, true>;
    return hmc_kernel<2, kWarpsPerBlock, false, true>;
  }
  return wpb == 8 ? hmc_kernel<3, 8, false, true> : hmc_kernel<3, kWarpsPerBlock, false, true>;
}
}  // namespace

size_t batch_smem_limit(int apl, int wpb, bool table) {
  int dev = 0, optin = 0;
  cudaFuncAttributes fa;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
      cudaFuncGetAttributes(&fa, batch_kernel(apl, wpb, table)) != cudaSuccess)
    return 0;
  return (size_t)optin > fa.sharedSizeBytes ? (size_t)optin - fa.sharedSizeBytes : 0;
}

bool batch_uses_table16(const LigandLayout& L) {
  const int apl = atoms_per_lane(L.na);
  return apl <= 2 && block_smem(L, apl, kTableWarps, true) <= batch_smem_limit(apl, kTableWarps, true);
}

cudaError_t batch_set_attributes(const algdock_ctx& c) {
  for (int k = 0; k < kBatchClasses; ++k) {
    const BatchClass& B = c.batch_cls[k];
    if (B.n_items == 0) continue;
    cudaError_t e = cudaFuncSetAttribute(batch_kernel(kClassApl[k], B.wpb, B.table),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B.smem);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One kernel per class (only_class >= 0: that class alone).  With more than one
// class the launches go to the context's side streams, forked from and joined back to s, so that
// they overlap (and capture into one graph with parallel branches).
cudaError_t launch_hmc_batch(cudaStream_t s, const algdock_ctx& c, const int32_t* state_of, float* x, double* comps,
                             double* dH, uint8_t* acc, int n_steps, uint64_t seed, uint64_t cycle, int64_t rep_offset,
                             int64_t* counters, int only_class) {
  HmcArgs A{c.grid, LigandLayout{}, c.d_batch_blob, c.d_states, c.K, c.batch_n_rep, state_of, x, comps, dH, acc,
            n_steps, seed, (uint32_t)cycle, rep_offset, counters, c.d_batch, nullptr, c.batch_x_stride, nullptr};
  int active[kBatchClasses], n_active = 0;
  for (int k = 0; k < kBatchClasses; ++k)
    if (c.batch_cls[k].n_items > 0 && (only_class < 0 || only_class == k)) active[n_active++] = k;
  if (n_active == 0) return cudaSuccess;
  cudaError_t e = cudaSuccess;
  if (n_active > 1) e = cudaEventRecord(c.batch_fork, s);
  for (int t = 0; t < n_active && e == cudaSuccess; ++t) {
    const int k = active[t];
    const BatchClass& B = c.batch_cls[k];
    cudaStream_t st = s;
    if (n_active > 1) {
      st = c.batch_side[k];
      e = cudaStreamWaitEvent(st, c.batch_fork, 0);
      if (e != cudaSuccess) break;
    }
    A.items = B.d_items;
    batch_kernel(kClassApl[k], B.wpb, B.table)<<<(unsigned)B.n_items, B.wpb * 32, B.smem, st>>>(A);
    e = cudaGetLastError();
    if (e == cudaSuccess && n_active > 1) {
      e = cudaEventRecord(c.batch_join[k], st);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(s, c.batch_join[k], 0);
    }
  }
  return e;
}

static cudaError_t launch_eval(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of,
                               const float* x, float* force, double* comps) {
  if (N == 0) return cudaSuccess;
  EvalArgs A{c.grid, c.lig, c.d_blob, c.d_states, c.K, N, state_of, x, force, comps};
  const int apl = atoms_per_lane(c.lig.na);
  if (force)
    return launch_templated(eval_kernel<1, true>, eval_kernel<2, true>, eval_kernel<3, true>, apl,
                            block_smem(c.lig, apl), N, s, A);
  return launch_templated(eval_kernel<1, false>, eval_kernel<2, false>, eval_kernel<3, false>, apl,
                          block_smem(c.lig, apl), N, s, A);
}

cudaError_t launch_evaluate(cudaStream_t s, const algdock_ctx& c, int64_t N, const float* x, double* comps) {
  return launch_eval(s, c, N, nullptr, x, nullptr, comps);
}

cudaError_t launch_energy_force(cudaStream_t s, const algdock_ctx& c, int64_t N, const int32_t* state_of,
                                const float* x, float* force, double* comps) {
  return launch_eval(s, c, N, state_of, x, force, comps);
}

cudaError_t launch_external(cudaStream_t s, const algdock_ctx& c, int64_t n_rep, const int32_t* state_of, float* x,
                            double* comps, int n_moves, double alpha_max, float sigma, uint64_t seed, uint64_t cycle,
                            int64_t rep_offset, int32_t* accepted, int64_t* counters) {
  if (n_rep == 0 || n_moves == 0) return cudaSuccess;
  ExtArgs A{c.grid, c.lig, c.d_blob, c.d_states, c.K, n_rep, state_of, x, comps, n_moves, alpha_max, sigma, seed,
            cycle, rep_offset, accepted, counters};
  const int apl = atoms_per_lane(c.lig.na);
  const unsigned blocks = (unsigned)((n_rep + kWarpsPerBlock - 1) / kWarpsPerBlock);
  if (apl == 1) external_kernel<1><<<blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else if (apl == 2) external_kernel<2><<<blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  else external_kernel<3><<<blocks, kWarpsPerBlock * 32, 0, s>>>(A);
  return cudaGetLastError();
}

cudaError_t launch_ukn(cudaStream_t s, const algdock_ctx& c, int64_t N, const double* comps, int k_begin,
                       int k_count, double* u_kn) {
  if (N == 0 || k_count == 0) return cudaSuccess;
  const int threads = 256;
  dim3 grid((unsigned)((N + threads - 1) / threads), (unsigned)min(k_count, 64));
  ukn_kernel<<<grid, threads, 0, s>>>(c.d_states, k_begin, k_count, N, comps, u_kn);
  return cudaGetLastError();
}

}  // namespace algdock
