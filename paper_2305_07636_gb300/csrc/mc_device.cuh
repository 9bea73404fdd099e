// Device building blocks of the random walk: Philox4x32-10, uniforms, particle state lanes,
// geometry distances, track-length DDA scoring, collision / surface / source sampling.
//
// The steps follow the problem statement of the MC/DC paper (Section 3: quadric CSG, multigroup,
// time-dependent source, time census, track-length mesh tallies, secondary production) with the
// textbook analog random walk; every random number comes from Philox4x32-10 (Salmon et al., SC'11)
// keyed by the run seed with the counter (particle tag, event index, block), so a history's
// random numbers do not depend on how the GPU schedules it.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "mc_internal.h"

namespace mcgb {

// ------------------------------------------------------------------------------------------ RNG
__device__ __forceinline__ uint4 philox4x32_10(uint32_t k0, uint32_t k1, uint4 c) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

template <typename R>
struct Uni;
// FP64: 52 random bits from the top 26 bits of two words, plus one half -> open interval (0,1)
template <>
struct Uni<double> {
  static __device__ __forceinline__ double from(uint32_t a, uint32_t b) {
    return (__uint2double_rn(a >> 6) * 67108864.0 + __uint2double_rn(b >> 6) + 0.5) *
           (1.0 / 4503599627370496.0);
  }
};
// FP32: 23 random bits of the first word plus one half -> open interval (0,1), exact in float:
// (m + 1/2) 2^-23 is formed as the float 1 + m 2^-23 (bit pattern) minus (1 - 2^-24); the
// subtraction is exact (Sterbenz), so no integer-to-float conversion is needed.
template <>
struct Uni<float> {
  static __device__ __forceinline__ float from(uint32_t a, uint32_t) {
    return __fsub_rn(__uint_as_float(0x3F800000u | (a >> 9)), 0.99999994039535522461f);
  }
};

template <typename R>
struct Pair2 {
  R a, b;
};

// two uniforms of block `blk` of event `k` of the particle tagged (tlo, thi)
template <typename R>
__device__ __forceinline__ Pair2<R> draw(uint64_t seed, uint32_t tlo, uint32_t thi, uint32_t k,
                                         uint32_t blk) {
  const uint4 r = philox4x32_10((uint32_t)seed, (uint32_t)(seed >> 32), make_uint4(tlo, thi, k, blk));
  return {Uni<R>::from(r.x, r.y), Uni<R>::from(r.z, r.w)};
}

__device__ __forceinline__ uint2 child_tag(uint64_t seed, uint32_t tlo, uint32_t thi, uint32_t k,
                                           uint32_t j, uint32_t mark) {
  const uint4 r = philox4x32_10((uint32_t)seed ^ kChildKeyXor, (uint32_t)(seed >> 32),
                                make_uint4(tlo, thi, k, mark | j));
  return make_uint2(r.x, r.y);
}

template <typename R>
__device__ __forceinline__ R rinf();
template <>
__device__ __forceinline__ float rinf<float>() { return CUDART_INF_F; }
template <>
__device__ __forceinline__ double rinf<double>() { return CUDART_INF; }

// a / b in the tracking precision: FP32 tracking takes the fast hardware divide (within 2 ulp; the
// correctly rounded one is a multi-instruction sequence and the walk divides several times per
// flight), FP64 tracking the correctly rounded one (the oracle's arithmetic, replayed to 1e-9)
__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float rlog(float u) { return __logf(u); }
// a * b and a + b rounded separately (never contracted into one FMA), as the oracle computes them
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rlog(double u) { return log(u); }
__device__ __forceinline__ float rsqrt_(float v) { return sqrtf(v); }
__device__ __forceinline__ double rsqrt_(double v) { return sqrt(v); }
// (cos 2 pi u, sin 2 pi u)
__device__ __forceinline__ void sincos2pi(float u, float* s, float* c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }

// true when i < n; in the bounds-checked build a false records MC_ERR_BOUNDS (first error wins)
__device__ __forceinline__ bool in_range(const RunParams& P, uint64_t i, uint64_t n) {
  if (!kChecked || i < n) return true;
  atomicCAS(&P.ctl->status, 0, MC_ERR_BOUNDS);
  atomicCAS(P.sticky, 0, MC_ERR_BOUNDS);
  return false;
}

// ------------------------------------------------------------------------------------------ tables
template <typename R>
struct Tab {
  const TableHeader* h;
  const R *st, *ss, *ssf, *nu, *nusf, *v, *inv_v, *scdf, *chi, *src_cdf, *scoef;
  const int *skind, *sbc, *nhs, *hs, *cmat, *cbox;
  const uint8_t* lpin;
  R lx0, ly0, lp, lr, lz0, lpz;
  int G;
  __device__ explicit Tab(const char* base) {
    h = reinterpret_cast<const TableHeader*>(base);
    st = reinterpret_cast<const R*>(base + h->o_st);
    ss = reinterpret_cast<const R*>(base + h->o_ss);
    ssf = reinterpret_cast<const R*>(base + h->o_ssf);
    nu = reinterpret_cast<const R*>(base + h->o_nu);
    nusf = reinterpret_cast<const R*>(base + h->o_nusf);
    v = reinterpret_cast<const R*>(base + h->o_v);
    inv_v = reinterpret_cast<const R*>(base + h->o_inv_v);
    scdf = reinterpret_cast<const R*>(base + h->o_scdf);
    chi = reinterpret_cast<const R*>(base + h->o_chi);
    src_cdf = reinterpret_cast<const R*>(base + h->o_src_cdf);
    scoef = reinterpret_cast<const R*>(base + h->o_scoef);
    skind = reinterpret_cast<const int*>(base + h->o_skind);
    sbc = reinterpret_cast<const int*>(base + h->o_sbc);
    nhs = reinterpret_cast<const int*>(base + h->o_nhs);
    hs = reinterpret_cast<const int*>(base + h->o_hs);
    cmat = reinterpret_cast<const int*>(base + h->o_cmat);
    cbox = reinterpret_cast<const int*>(base + h->o_cbox);
    lpin = reinterpret_cast<const uint8_t*>(base + h->o_lpin);
    lx0 = (R)h->lat_x0;
    ly0 = (R)h->lat_y0;
    lp = (R)h->lat_pitch;
    lr = (R)h->lat_r;
    lz0 = (R)h->lat_z0;
    lpz = (R)h->lat_pz;
    G = h->G;
  }
};

// ------------------------------------------------------------------------------------------ state
// Particle time.  FP64 tracking keeps a double (the oracle's arithmetic).  FP32 tracking keeps
// an unevaluated sum of two floats (hi + lo): additions use the exact two-sum of Knuth, so the
// clock carries about 48 significant bits and the census comparison keeps FP64-class resolution
// without the FP64 pipe, which on this GPU runs at 1/64 of the FP32 rate.
template <typename R>
struct Part;

template <>
struct Part<float> {
  float x, y, z, ux, uy, uz;
  float th, tl;  // time = th + tl
  double w;
  uint32_t tlo, thi, k, pk, elem, root;
  __device__ __forceinline__ float time() const { return th + tl; }
  __device__ __forceinline__ void zero_time() { th = tl = 0.0f; }
  __device__ __forceinline__ double time_d() const { return (double)th + (double)tl; }
  __device__ __forceinline__ void advance(float l, float v, float inv_v) {
    const float b = __fmul_rn(l, inv_v);
    const float s = __fadd_rn(th, b);
    const float bb = __fsub_rn(s, th);
    const float err = __fadd_rn(__fsub_rn(th, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    const float lo = __fadd_rn(tl, err);
    th = __fadd_rn(s, lo);
    tl = __fsub_rn(lo, __fsub_rn(th, s));
  }
  // v (t_census - t), with the census time given as hi + lo
  __device__ __forceinline__ float census_distance(float tch, float tcl, float v) const {
    return __fadd_rn(__fsub_rn(tch, th), __fsub_rn(tcl, tl)) * v;
  }
};

template <>
struct Part<double> {
  double x, y, z, ux, uy, uz;
  double t;
  double w;
  uint32_t tlo, thi, k, pk, elem, root;
  __device__ __forceinline__ double time() const { return t; }
  __device__ __forceinline__ void zero_time() { t = 0.0; }
  __device__ __forceinline__ double time_d() const { return t; }
  __device__ __forceinline__ void advance(double l, double v, double) { t += l / v; }
  __device__ __forceinline__ double census_distance(double tc, double, double v) const {
    return v * (tc - t);
  }
};

// packed 16-byte lanes; the same layout in global banks and in the shared-memory queue
template <typename R>
struct Lanes;

// FP32 particle = 4 x 16 B: (x,y,z,ux) (uy,uz,elem,root) (t_hi,t_lo,w) (tag_lo,tag_hi,k,packed)
template <>
struct Lanes<float> {
  static constexpr int N = kLanesFP32;
  static __device__ __forceinline__ void pack(const Part<float>& p, uint4 v[N]) {
    v[0] = make_uint4(__float_as_uint(p.x), __float_as_uint(p.y), __float_as_uint(p.z), __float_as_uint(p.ux));
    v[1] = make_uint4(__float_as_uint(p.uy), __float_as_uint(p.uz), p.elem, p.root);
    const unsigned long long wb = (unsigned long long)__double_as_longlong(p.w);
    v[2] = make_uint4(__float_as_uint(p.th), __float_as_uint(p.tl), (uint32_t)wb, (uint32_t)(wb >> 32));
    v[3] = make_uint4(p.tlo, p.thi, p.k, p.pk);
  }
  static __device__ __forceinline__ void unpack(const uint4 v[N], Part<float>& p) {
    p.x = __uint_as_float(v[0].x); p.y = __uint_as_float(v[0].y); p.z = __uint_as_float(v[0].z);
    p.ux = __uint_as_float(v[0].w); p.uy = __uint_as_float(v[1].x); p.uz = __uint_as_float(v[1].y);
    p.elem = v[1].z; p.root = v[1].w;
    p.th = __uint_as_float(v[2].x); p.tl = __uint_as_float(v[2].y);
    p.w = __longlong_as_double((long long)(((unsigned long long)v[2].w << 32) | v[2].z));
    p.tlo = v[3].x; p.thi = v[3].y; p.k = v[3].z; p.pk = v[3].w;
  }
};

// FP64 particle = 6 x 16 B: (x,y) (z,ux) (uy,uz) (t,w) (tag_lo,tag_hi,k,packed) (elem,root,-,-)
template <>
struct Lanes<double> {
  static constexpr int N = kLanesFP64;
  static __device__ __forceinline__ uint4 d2(double a, double b) {
    const unsigned long long x = (unsigned long long)__double_as_longlong(a);
    const unsigned long long y = (unsigned long long)__double_as_longlong(b);
    return make_uint4((uint32_t)x, (uint32_t)(x >> 32), (uint32_t)y, (uint32_t)(y >> 32));
  }
  static __device__ __forceinline__ double lo(const uint4& v) {
    return __longlong_as_double((long long)(((unsigned long long)v.y << 32) | v.x));
  }
  static __device__ __forceinline__ double hi(const uint4& v) {
    return __longlong_as_double((long long)(((unsigned long long)v.w << 32) | v.z));
  }
  static __device__ __forceinline__ void pack(const Part<double>& p, uint4 v[N]) {
    v[0] = d2(p.x, p.y);
    v[1] = d2(p.z, p.ux);
    v[2] = d2(p.uy, p.uz);
    v[3] = d2(p.t, p.w);
    v[4] = make_uint4(p.tlo, p.thi, p.k, p.pk);
    v[5] = make_uint4(p.elem, p.root, 0u, 0u);
  }
  static __device__ __forceinline__ void unpack(const uint4 v[N], Part<double>& p) {
    p.x = lo(v[0]); p.y = hi(v[0]); p.z = lo(v[1]); p.ux = hi(v[1]); p.uy = lo(v[2]); p.uz = hi(v[2]);
    p.t = lo(v[3]); p.w = hi(v[3]);
    p.tlo = v[4].x; p.thi = v[4].y; p.k = v[4].z; p.pk = v[4].w;
    p.elem = v[5].x; p.root = v[5].y;
  }
};

// Global bank access: 16-byte vector loads and stores, lane-major SoA.  Loads go through L2 only
// (ld.global.cg): the banks are rewritten by other SMs between grid-barrier iterations and the
// per-SM L1 is not coherent, so an L1-cached load could return a line from an earlier iteration.
// Each slot is read once per iteration, so L1 would not help anyway.
template <typename R>
__device__ __forceinline__ void bank_load(Part<R>& p, uint4* const* L, uint64_t i) {
  uint4 v[Lanes<R>::N];
#pragma unroll
  for (int l = 0; l < Lanes<R>::N; ++l) v[l] = __ldcg(L[l] + i);
  Lanes<R>::unpack(v, p);
}
template <typename R>
__device__ __forceinline__ void bank_store(const Part<R>& p, uint4* const* L, uint64_t i) {
  uint4 v[Lanes<R>::N];
  Lanes<R>::pack(p, v);
#pragma unroll
  for (int l = 0; l < Lanes<R>::N; ++l) __stcs(L[l] + i, v[l]);
}
// shared-memory queue access: lane l of slot i at q[l * cap + i]
template <typename R>
__device__ __forceinline__ void queue_load(Part<R>& p, const uint4* q, unsigned cap, unsigned i) {
  uint4 v[Lanes<R>::N];
#pragma unroll
  for (int l = 0; l < Lanes<R>::N; ++l) v[l] = q[l * cap + i];
  Lanes<R>::unpack(v, p);
}
template <typename R>
__device__ __forceinline__ void queue_store(const Part<R>& p, uint4* q, unsigned cap, unsigned i) {
  uint4 v[Lanes<R>::N];
  Lanes<R>::pack(p, v);
#pragma unroll
  for (int l = 0; l < Lanes<R>::N; ++l) q[l * cap + i] = v[l];
}

// the time of a particle set to the launch's census time exactly (population-control copies)
__device__ __forceinline__ void set_census_time(Part<float>& p, const RunParams& P) {
  p.th = P.tc_hi;
  p.tl = P.tc_lo;
}
__device__ __forceinline__ void set_census_time(Part<double>& p, const RunParams& P) { p.t = P.tc; }

// Fission sites of a k-eigenvalue cycle (position and group): FP32 one 16-byte vector (x, y, z, g),
// FP64 two ((x, y), (z, g)), at index i of a site array
__device__ __forceinline__ void site_store(uint4* a, uint64_t i, float x, float y, float z, int g) {
  a[i] = make_uint4(__float_as_uint(x), __float_as_uint(y), __float_as_uint(z), (uint32_t)g);
}
__device__ __forceinline__ void site_store(uint4* a, uint64_t i, double x, double y, double z, int g) {
  const unsigned long long bx = (unsigned long long)__double_as_longlong(x), by = (unsigned long long)__double_as_longlong(y),
                           bz = (unsigned long long)__double_as_longlong(z);
  a[2 * i] = make_uint4((uint32_t)bx, (uint32_t)(bx >> 32), (uint32_t)by, (uint32_t)(by >> 32));
  a[2 * i + 1] = make_uint4((uint32_t)bz, (uint32_t)(bz >> 32), (uint32_t)g, 0u);
}
__device__ __forceinline__ void site_load(const uint4* a, uint64_t i, float& x, float& y, float& z, int& g) {
  const uint4 v = __ldcg(a + i);
  x = __uint_as_float(v.x);
  y = __uint_as_float(v.y);
  z = __uint_as_float(v.z);
  g = (int)v.w;
}
__device__ __forceinline__ void site_load(const uint4* a, uint64_t i, double& x, double& y, double& z, int& g) {
  const uint4 v = __ldcg(a + 2 * i), w = __ldcg(a + 2 * i + 1);
  x = __longlong_as_double((long long)(((unsigned long long)v.y << 32) | v.x));
  y = __longlong_as_double((long long)(((unsigned long long)v.w << 32) | v.z));
  z = __longlong_as_double((long long)(((unsigned long long)w.y << 32) | w.x));
  g = (int)w.z;
}

// Round-to-nearest double -> float on the integer pipes (positive normal weights; smaller
// magnitudes flush to 0, larger saturate to infinity).  The hardware conversion runs on the slow
// FP64 pipe of this GPU.
__device__ __forceinline__ float weight_to_float(double w) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(w) + (1ull << 28);
  const int e = (int)((b >> 52) & 0x7FF) - 1023;
  if (e < -126) return 0.0f;
  if (e > 127) return CUDART_INF_F;
  return __uint_as_float(((uint32_t)(e + 127) << 23) | (uint32_t)((b >> 29) & 0x7FFFFFu));
}

// Non-negative float -> nearest int64 (ties up), from the float's bits: the hardware float-to-
// int64 conversion also runs on the slow FP64 pipe.
__device__ __forceinline__ long long float_to_fixed(float f) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)(b >> 23) - 127;  // f = 1.m 2^e
  if ((b >> 31) || e < -1) return 0ll;
  const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
  if (e >= 23) return e >= 62 ? 0x7FFFFFFFFFFFFFFFll : (long long)(m << (e - 23));
  const int sh = 23 - e;  // 1 .. 24
  return (long long)((m + (1ull << (sh - 1))) >> sh);
}

// ------------------------------------------------------------------------------------------ geometry
// lattice element index e = (iz ny + iy) nx + ix in the low 16 bits of the elem word
__device__ __forceinline__ uint32_t lat_e(uint32_t elem) { return elem & 0xFFFFu; }
__device__ __forceinline__ uint32_t lat_pack(uint32_t elem, uint32_t e) { return (elem & 0xFFFF0000u) | e; }

struct LatIdx {
  int ix, iy, iz;
};
// (ix, iy, iz) of element e: n / d = floor(n ceil(2^32 / d) / 2^32) exactly for n < 2^16 and
// d <= 2^16 (the rounding-up error of the reciprocal adds less than n / 2^32 < 1 / d)
template <typename R>
__device__ __forceinline__ LatIdx lat_split(const Tab<R>& T, uint32_t e) {
  const uint32_t q = (uint32_t)(((unsigned long long)e * T.h->lat_mx) >> 32);
  const uint32_t iz = (uint32_t)(((unsigned long long)q * T.h->lat_my) >> 32);
  return {(int)(e - q * (uint32_t)T.h->lat_nx), (int)(q - iz * (uint32_t)T.h->lat_ny), (int)iz};
}

template <typename R>
__device__ __forceinline__ int material_of(const Tab<R>& T, uint32_t pk, uint32_t elem) {
  const int m = T.cmat[pk_cell(pk)];
  if (m >= 0) return m;
  if (pk_pin(pk)) return (int)T.lpin[lat_e(elem)];
  return T.h->lat_matrix;
}

// distance to a plane, counted only while the motion leaves the half-space (sense +1: f >= 0)
template <typename R>
__device__ __forceinline__ R plane_dist(R pos, R u, R c, int sense) {
  const bool leaving = sense > 0 ? (u < R(0)) : (u > R(0));
  if (!leaving) return rinf<R>();
  const R d = rdiv(c - pos, u);
  return d > R(0) ? d : R(0);
}

// distance to a z-cylinder: from inside the far root, from outside the near root when approaching
template <typename R>
__device__ __forceinline__ R cyl_dist(R x, R y, R ux, R uy, R x0, R y0, R r, bool inside) {
  const R a = ux * ux + uy * uy;
  if (a == R(0)) return rinf<R>();
  const R dx = x - x0, dy = y - y0;
  const R b = dx * ux + dy * uy;
  const R c = dx * dx + dy * dy - r * r;
  R disc = b * b - a * c;
  if (inside) {
    if (disc < R(0)) disc = R(0);
    const R sq = rsqrt_(disc);
    const R d = (b <= R(0)) ? rdiv(-b + sq, a) : rdiv(-c, b + sq);
    return d > R(0) ? d : R(0);
  }
  if (b >= R(0) || disc <= R(0)) return rinf<R>();
  // A grazing line whose chord inside the cylinder, 2 sqrt(disc) / a, is shorter than eps does
  // not enter it: otherwise rounding can put a tangentially moving particle inside with a zero
  // exit distance and bounce it in and out on the spot.  eps = 2e-5 cm (FP32), 1e-12 cm (FP64).
  const R sq = rsqrt_(disc);
  if (R(2) * sq < (sizeof(R) == 4 ? R(2e-5) : R(1e-12)) * a) return rinf<R>();
  const R d = rdiv(c, -b + sq);
  return d > R(0) ? d : R(0);
}

// A quadric surface (cylinders along x or y, spheres, general quadrics) along the ray p + t u:
// f(t) = a t^2 + b t + c, with the quadric A..J written about its centre: (X, Y, Z) = p - centre.
template <typename R>
__device__ __forceinline__ void quad_ray(const R* k, R x, R y, R z, R ux, R uy, R uz, R& a, R& b, R& c) {
  const R* q = k + 3;
  const R X = x - k[13], Y = y - k[14], Z = z - k[15];
  a = q[0] * ux * ux + q[1] * uy * uy + q[2] * uz * uz + q[3] * ux * uy + q[4] * uy * uz + q[5] * uz * ux;
  b = R(2) * (q[0] * X * ux + q[1] * Y * uy + q[2] * Z * uz) + q[3] * (X * uy + Y * ux) + q[4] * (Y * uz + Z * uy) +
      q[5] * (Z * ux + X * uz) + q[6] * ux + q[7] * uy + q[8] * uz;
  c = q[0] * X * X + q[1] * Y * Y + q[2] * Z * Z + q[3] * X * Y + q[4] * Y * Z + q[5] * Z * X + q[6] * X + q[7] * Y +
      q[8] * Z + q[9];
}

// Distance at which the particle leaves its half-space of a quadric (sense +1: f >= 0, -1: f < 0):
// the root of f(t) where f falls (sense +1) or rises (sense -1).  A root just behind counts as 0
// where the particle is on the surface heading out of a convex section; a grazing entry into a convex
// section whose chord sqrt(disc) / a is shorter than eps (2e-5 cm FP32, 1e-12 cm FP64) is no crossing.
template <typename R>
__device__ __forceinline__ R dist_quadric(R a, R b, R c, int sense) {
  if (a == R(0)) {
    if (b == R(0) || (sense > 0) == (b > R(0))) return rinf<R>();  // f linear along the ray, not leaving
    const R t = rdiv(-c, b);
    return t > R(0) ? t : R(0);
  }
  R disc = b * b - R(4) * a * c;
  if (sense < 0) {  // the root where f rises
    if (disc < R(0)) {
      if (a > R(0)) disc = R(0);  // inside a convex section: rounding
      else return rinf<R>();
    }
    const R sq = rsqrt_(disc);
    const R t = b <= R(0) ? rdiv(-b + sq, R(2) * a) : rdiv(R(-2) * c, b + sq);
    if (!(t > R(0))) return a > R(0) ? R(0) : rinf<R>();
    return t;
  }
  if (disc <= R(0)) return rinf<R>();  // the root where f falls
  const R sq = rsqrt_(disc);
  if (a > R(0) && sq < (sizeof(R) == 4 ? R(2e-5) : R(1e-12)) * a) return rinf<R>();
  const R t = b >= R(0) ? rdiv(-b - sq, R(2) * a) : rdiv(R(-2) * c, b - sq);
  if (!(t > R(0))) return (a > R(0) && b < R(0)) ? R(0) : rinf<R>();
  return t;
}

template <typename R>
__device__ __forceinline__ R surf_f(const Tab<R>& T, int s, R x, R y, R z) {
  const R* c = T.scoef + kSurfStride * s;
  switch (T.skind[s]) {
    case MC_SURF_PX: return x - c[0];
    case MC_SURF_PY: return y - c[0];
    case MC_SURF_PZ: return z - c[0];
    case MC_SURF_CZ: {
      const R dx = x - c[0], dy = y - c[1];
      return dx * dx + dy * dy - c[2] * c[2];
    }
    default: {
      R a, b, f;
      quad_ray(c, x, y, z, R(0), R(0), R(0), a, b, f);
      return f;
    }
  }
}

// rounding scale of surf_f at a point: the magnitude of the terms it subtracts
template <typename R>
__device__ __forceinline__ R surf_scale(const Tab<R>& T, int s, R x, R y, R z) {
  const R* c = T.scoef + kSurfStride * s;
  switch (T.skind[s]) {
    case MC_SURF_PX: return R(1) + fabs(x) + fabs(c[0]);
    case MC_SURF_PY: return R(1) + fabs(y) + fabs(c[0]);
    case MC_SURF_PZ: return R(1) + fabs(z) + fabs(c[0]);
    case MC_SURF_CZ: {
      const R dx = x - c[0], dy = y - c[1];
      return R(1) + dx * dx + dy * dy + c[2] * c[2];
    }
    default: {
      const R* q = c + 3;
      const R X = x - c[13], Y = y - c[14], Z = z - c[15];
      return R(1) + fabs(q[0] * X * X) + fabs(q[1] * Y * Y) + fabs(q[2] * Z * Z) + fabs(q[3] * X * Y) +
             fabs(q[4] * Y * Z) + fabs(q[5] * Z * X) + fabs(q[6] * X) + fabs(q[7] * Y) + fabs(q[8] * Z) + fabs(q[9]);
    }
  }
}

// normal component of the direction on surface s (the side a point on s is moving into)
template <typename R>
__device__ __forceinline__ R surf_dir(const Tab<R>& T, int s, R x, R y, R z, R ux, R uy, R uz) {
  const R* c = T.scoef + kSurfStride * s;
  switch (T.skind[s]) {
    case MC_SURF_PX: return ux;
    case MC_SURF_PY: return uy;
    case MC_SURF_PZ: return uz;
    case MC_SURF_CZ: return (x - c[0]) * ux + (y - c[1]) * uy;
    default: {
      R a, b, f;
      quad_ray(c, x, y, z, ux, uy, uz, a, b, f);
      return b;  // the rate at which f changes along the direction
    }
  }
}

// First cell containing the point.  If skip >= 0 the point was reached by crossing surface
// `skip`: the half-space on it is taken to have sense `skip_sense` without evaluating it, and the
// other half-spaces are tested with the direction (ux, uy, uz):
//  - a point exactly on another surface (f == 0, e.g. a corner where the crossed plane meets a
//    second one) is on the side the direction points into (the + side when moving along it);
//    the plain f >= 0 convention could send such a particle back and forth between two cells in
//    zero-length flights forever;
//  - if no cell contains the point, one that contains it within the rounding tolerance (1e-5
//    relative in FP32, 1e-12 in FP64, of surf_scale) is taken, the first in cell order: a
//    crossing next to a reflecting wall can round to just outside the wall.
// Without a crossing (skip < 0) a point on a surface is on its + side.
template <typename R>
__device__ int locate_cell(const Tab<R>& T, R x, R y, R z, int skip, int skip_sense, R ux = R(0), R uy = R(0),
                           R uz = R(0)) {
  const R eps = sizeof(R) == 4 ? R(1e-5) : R(1e-12);
  for (int pass = 0; pass < (skip >= 0 ? 2 : 1); ++pass) {
    for (int c = 0; c < T.h->n_cell; ++c) {
      bool ok = true, seen = skip < 0;
      const int n = T.nhs[c];
      for (int i = 0; i < n && ok; ++i) {
        const int e = T.hs[c * MC_MAX_HALFSPACES + i];
        const int s = e & 0xFFFF, sn = (e >> 16) ? -1 : 1;
        if (s == skip) {
          seen = true;
          ok = sn == skip_sense;
        } else {
          const R f = surf_f(T, s, x, y, z);
          if (pass == 0) {
            const R d = f != R(0) ? f : surf_dir(T, s, x, y, z, ux, uy, uz);
            ok = sn > 0 ? (d >= R(0)) : (d < R(0));
          } else {
            const R tol = eps * surf_scale(T, s, x, y, z);
            ok = sn > 0 ? (f >= -tol) : (f < tol);
          }
        }
      }
      if (ok && seen) return c;
    }
  }
  return -1;
}

template <typename R>
__device__ __forceinline__ uint32_t pin_inside(const Tab<R>& T, R x, R y, int ix, int iy, uint32_t e) {
  if (T.lpin[e] == kNoPin) return 0u;
  const R dx = x - (T.lx0 + (R(ix) + R(0.5)) * T.lp), dy = y - (T.ly0 + (R(iy) + R(0.5)) * T.lp);
  return (dx * dx + dy * dy - T.lr * T.lr) < R(0) ? 1u : 0u;
}

// lattice element and pin sense of a point inside the lattice cell
template <typename R>
__device__ __forceinline__ void lattice_locate(const Tab<R>& T, Part<R>& p) {
  int ix = (int)floor((p.x - T.lx0) / T.lp), iy = (int)floor((p.y - T.ly0) / T.lp), iz = 0;
  ix = min(max(ix, 0), T.h->lat_nx - 1);
  iy = min(max(iy, 0), T.h->lat_ny - 1);
  if (T.h->lat_nz > 1) {
    iz = (int)floor((p.z - T.lz0) / T.lpz);
    iz = min(max(iz, 0), T.h->lat_nz - 1);
  }
  const uint32_t e = (uint32_t)((iz * T.h->lat_ny + iy) * T.h->lat_nx + ix);
  p.elem = lat_pack(p.elem, e);
  p.pk = (p.pk & ~(1u << 13)) | (pin_inside(T, p.x, p.y, ix, iy, e) << 13);
}

struct Hit {
  uint32_t type;
  int dir;
  uint32_t surf;
  uint32_t chan;  // channel of a collision at the end of the flight (CHAN_*)
};

// Cells bounded by axis-aligned planes only take a shortcut of the surface loop (the same
// distances and choice); a translation unit that sets MCGB_BOX_CELLS to 0 compiles the loop alone.
#ifndef MCGB_BOX_CELLS
#define MCGB_BOX_CELLS 1
#endif
template <typename R>
__device__ R boundary_distance(const Tab<R>& T, const Part<R>& p, Hit& hit) {
  R best = rinf<R>();
  hit = {HIT_CELL, 1, 0};
  const int c = (int)pk_cell(p.pk);
  const int n = MCGB_BOX_CELLS && T.cbox[7 * c] ? 0 : T.nhs[c];
  if (MCGB_BOX_CELLS && n == 0) {
    // a box cell: per axis only the plane the motion can leave by, with the generic loop's
    // distance expression and its choice among equal distances (the earliest in the cell's list)
    const int* bx = T.cbox + 7 * c + 1;
    const R pos[3] = {p.x, p.y, p.z}, u[3] = {p.ux, p.uy, p.uz};
    int bo = 1 << 30;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const int e = u[a] > R(0) ? bx[2 * a + 1] : (u[a] < R(0) ? bx[2 * a] : -1);
      if (e >= 0) {
        const int s = e & 0xFFFF, o = e >> 16;
        R d = rdiv(T.scoef[kSurfStride * s] - pos[a], u[a]);
        d = d > R(0) ? d : R(0);
        if (d < best || (d == best && d < rinf<R>() && o < bo)) {
          best = d;
          bo = o;
          hit = {HIT_CELL, 1, (uint32_t)s};
        }
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    const int e = T.hs[c * MC_MAX_HALFSPACES + i];
    const int s = e & 0xFFFF, sn = (e >> 16) ? -1 : 1;
    const R* cf = T.scoef + kSurfStride * s;
    R d;
    switch (T.skind[s]) {
      case MC_SURF_PX: d = plane_dist(p.x, p.ux, cf[0], sn); break;
      case MC_SURF_PY: d = plane_dist(p.y, p.uy, cf[0], sn); break;
      case MC_SURF_PZ: d = plane_dist(p.z, p.uz, cf[0], sn); break;
      case MC_SURF_CZ: d = cyl_dist(p.x, p.y, p.ux, p.uy, cf[0], cf[1], cf[2], sn < 0); break;
      default: {
        R a, b, f;
        quad_ray(cf, p.x, p.y, p.z, p.ux, p.uy, p.uz, a, b, f);
        d = dist_quadric(a, b, f, sn);
        break;
      }
    }
    if (d < best) {
      best = d;
      hit = {HIT_CELL, 1, (uint32_t)s};
    }
  }
  if (T.cmat[c] < 0) {
    // lattice: inner element walls in the direction of motion (x, y, then z between axial
    // layers), then the pin; the hit's surf field carries the wall's axis
    const uint32_t e = lat_e(p.elem);
    const LatIdx L = lat_split(T, e);
    const int ix = L.ix, iy = L.iy;
    const R xlo = T.lx0 + R(ix) * T.lp, ylo = T.ly0 + R(iy) * T.lp;
    R lbest = rinf<R>();
    Hit lh = {HIT_LAT, 1, 0};
    if (p.ux > R(0) && ix + 1 < T.h->lat_nx) {
      R d = rdiv(xlo + T.lp - p.x, p.ux);
      d = d > R(0) ? d : R(0);
      if (d < lbest) { lbest = d; lh = {HIT_LAT, 1, 0}; }
    } else if (p.ux < R(0) && ix > 0) {
      R d = rdiv(xlo - p.x, p.ux);
      d = d > R(0) ? d : R(0);
      if (d < lbest) { lbest = d; lh = {HIT_LAT, -1, 0}; }
    }
    if (p.uy > R(0) && iy + 1 < T.h->lat_ny) {
      R d = rdiv(ylo + T.lp - p.y, p.uy);
      d = d > R(0) ? d : R(0);
      if (d < lbest) { lbest = d; lh = {HIT_LAT, 1, 1}; }
    } else if (p.uy < R(0) && iy > 0) {
      R d = rdiv(ylo - p.y, p.uy);
      d = d > R(0) ? d : R(0);
      if (d < lbest) { lbest = d; lh = {HIT_LAT, -1, 1}; }
    }
    if (T.h->lat_nz > 1) {
      const R zlo = T.lz0 + R(L.iz) * T.lpz;
      if (p.uz > R(0) && L.iz + 1 < T.h->lat_nz) {
        R d = rdiv(zlo + T.lpz - p.z, p.uz);
        d = d > R(0) ? d : R(0);
        if (d < lbest) { lbest = d; lh = {HIT_LAT, 1, 2}; }
      } else if (p.uz < R(0) && L.iz > 0) {
        R d = rdiv(zlo - p.z, p.uz);
        d = d > R(0) ? d : R(0);
        if (d < lbest) { lbest = d; lh = {HIT_LAT, -1, 2}; }
      }
    }
    if (T.lpin[e] != kNoPin) {
      const R d = cyl_dist(p.x, p.y, p.ux, p.uy, xlo + R(0.5) * T.lp, ylo + R(0.5) * T.lp, T.lr,
                           pk_pin(p.pk) != 0);
      if (d < lbest) { lbest = d; lh = {HIT_PIN, 1, 0}; }
    }
    if (lbest < best) {
      best = lbest;
      hit = lh;
    }
  }
  return best;
}

// i with e[i] <= x < e[i+1] over n bins; -1 below the first edge, n at or above the last
template <typename E, typename X>
__device__ __forceinline__ int bin_search(const E* e, int n, X x) {
  if (!(x >= (X)e[0])) return -1;
  if (!(x < (X)e[n])) return n;
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((X)e[mid] <= x) lo = mid;
    else hi = mid;
  }
  return lo;
}

// The same bin as bin_search, from a first guess along an axis of equal (kind 1) or geometric
// (kind 2, from edge 1 on) spacing, corrected against the edges: the guess lands within a bin of
// the answer, and the walk to e[i] <= x < e[i+1] settles the rounding of the guess.  Kind 0 is
// plain bisection.  The segment walk of the persistent kernel starts with it; the batched
// kernel's translation unit sets MCGB_BIN_GUESS to 0 and keeps bisection (that kernel is bound by
// instruction fetch, and the guess's code measured slower there).
#ifndef MCGB_BIN_GUESS
#define MCGB_BIN_GUESS 1
#endif
__device__ __forceinline__ int bin_find(const float* e, int n, float x, int kind, float a, float b) {
  if (kind == 0) return bin_search(e, n, x);
  if (!(x >= e[0])) return -1;
  if (!(x < e[n])) return n;
  int i;
  if (kind == 1) i = __float2int_rd(__fmul_rn(__fsub_rn(x, a), b));
  else i = x < e[1] ? 0 : 1 + __float2int_rd(__fmul_rn(__log2f(__fmul_rn(x, a)), b));
  i = min(max(i, 0), n - 1);
  while (i > 0 && x < e[i]) --i;
  while (i < n - 1 && !(x < e[i + 1])) ++i;
  return i;
}

// ------------------------------------------------------------------------------------------ tally atomics
__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// Warp-aggregated add: lanes that target the same bin are found with match.any; each peer group
// is reduced by a shuffle tree over the group's ranks and its lowest lane issues one atomic.  The
// tree runs only as deep as the largest group needs, so a warp without shared bins pays one
// match and one vote.
template <typename V>
__device__ __forceinline__ V peer_reduce(unsigned mask, unsigned peers, V v, unsigned depth) {
  const int lane = threadIdx.x & 31;
  const unsigned rank = __popc(peers & lanemask_lt());
  for (unsigned d = 1; d < depth; d <<= 1) {
    const unsigned src = __fns(peers, (unsigned)lane, (int)d + 1);
    const V o = __shfl_sync(mask, v, (src == 0xFFFFFFFFu) ? lane : (int)src);
    if (src != 0xFFFFFFFFu && (rank & (2 * d - 1)) == 0) v += o;
  }
  return v;
}

// tally adds whose old value nobody reads: reductions (no value comes back from L2)
__device__ __forceinline__ void red_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.global.add.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v) : "memory");
}
__device__ __forceinline__ void red_add(double* p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "d"(v) : "memory");
}

__device__ __forceinline__ void add_fixed(unsigned long long* dst, long long v, bool aggregate) {
  if (aggregate) {
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, (unsigned long long)dst);
    const unsigned depth = __reduce_max_sync(mask, (unsigned)__popc(peers));
    if (depth > 1) v = peer_reduce(mask, peers, v, depth);
    if ((peers & lanemask_lt()) == 0u) red_add(dst, (unsigned long long)v);
  } else {
    red_add(dst, (unsigned long long)v);
  }
}

__device__ __forceinline__ void add_fp64(double* dst, double v, bool aggregate) {
  if (aggregate) {
    const unsigned mask = __activemask();
    const unsigned peers = __match_any_sync(mask, (unsigned long long)dst);
    const unsigned depth = __reduce_max_sync(mask, (unsigned)__popc(peers));
    if (depth > 1) v = peer_reduce(mask, peers, v, depth);
    if ((peers & lanemask_lt()) == 0u) red_add(dst, v);
  } else {
    red_add(dst, v);
  }
}

// Scorer for one flight: the weight factor is converted once per flight, not per piece.
template <typename R>
struct Scorer {
  const RunParams& P;
  double w;        // FP64 tallies
  float wscale;    // fixed-point tallies: w * 2^bits
  __device__ Scorer(const RunParams& P_, double w_)
      : P(P_), w(w_), wscale(sizeof(R) == 4 ? weight_to_float(w_) * P_.fixed_scale_f : 0.0f) {}
  __device__ __forceinline__ void operator()(uint64_t slot, R len) const {
    if (!in_range(P, slot, (uint64_t)P.tally_stripes * P.stripe_stride)) return;
    if (P.tally_fp64) {
      add_fp64(reinterpret_cast<double*>(P.tally) + slot, w * (double)len, P.aggregate != 0);
    } else {
      const long long q = sizeof(R) == 4 ? float_to_fixed(wscale * (float)len)
                                         : __double2ll_rn(w * (double)len * P.fixed_scale);
      add_fixed(reinterpret_cast<unsigned long long*>(P.tally) + slot, q, P.aggregate != 0);
    }
  }
};

template <typename R>
__device__ __forceinline__ const R* time_edges(const char* base, const TallyDesc& D);
template <>
__device__ __forceinline__ const float* time_edges<float>(const char* base, const TallyDesc& D) {
  return reinterpret_cast<const float*>(base + D.o_etf);
}
template <>
__device__ __forceinline__ const double* time_edges<double>(const char* base, const TallyDesc& D) {
  return reinterpret_cast<const double*>(base + D.o_et);
}

// Per-warp staging buffer of tally scores in shared memory: slot index and the score's bits
// (int64 fixed point or double).
struct Stage {
  uint32_t* slot;
  unsigned long long* val;
};

// Adds the n staged scores with all 32 lanes converged, 32 at a time, so that the match-based
// warp aggregation sees whole warps.  Must be called by all lanes with a warp-uniform n.
__device__ __forceinline__ void stage_flush(const RunParams& P, const Stage& S, unsigned n) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  for (unsigned b = 0; b < n; b += 32) {
    const unsigned i = b + lane;
    if (i < n) {
      const uint32_t slot = S.slot[i];
      const unsigned long long v = S.val[i];
      if (!in_range(P, slot, (uint64_t)P.tally_stripes * P.stripe_stride)) continue;
      if (P.tally_fp64)
        add_fp64(reinterpret_cast<double*>(P.tally) + slot, __longlong_as_double((long long)v), P.aggregate != 0);
      else
        add_fixed(reinterpret_cast<unsigned long long*>(P.tally) + slot, (long long)v, P.aggregate != 0);
    }
  }
  __syncwarp();
}

// Score bits of a piece in the modes that need FP64 arithmetic (FP64 tallies, or fixed point
// with FP64 tracking).  Not inlined, so that the FP32 fixed-point path carries no FP64 pipe work
// (this GPU runs FP64 at 1/64 of the FP32 rate).
static __device__ __noinline__ unsigned long long score_bits_fp64(const RunParams& P, double w, double len) {
  if (P.tally_fp64) return (unsigned long long)__double_as_longlong(w * len);
  return (unsigned long long)__double2ll_rn(w * len * P.fixed_scale);
}

template <typename R>
struct ScoreSink {
  const RunParams& P;
  const Stage& S;
  unsigned& pieces;
  unsigned n_st;
  double w;
  float wscale;
  __device__ ScoreSink(const RunParams& P_, const Stage& S_, unsigned& pieces_, double w_)
      : P(P_), S(S_), pieces(pieces_), n_st(0u), w(w_),
        wscale(sizeof(R) == 4 ? weight_to_float(w_) * P_.fixed_scale_f : 0.0f) {}
  __device__ __forceinline__ void add(bool emit, uint32_t slot, R len) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, emit);
    unsigned long long val = 0ull;
    if (emit) {
      if (sizeof(R) == 4 && !P.tally_fp64) {
        const long long qv = float_to_fixed(wscale * fabsf((float)len));
        val = (unsigned long long)(len < R(0) ? -qv : qv);
      } else {
        val = score_bits_fp64(P, w, (double)len);
      }
    }
    pieces += __popc(m);
    if (!P.aggregate) {
      if (emit && in_range(P, slot, (uint64_t)P.tally_stripes * P.stripe_stride)) {
        if (P.tally_fp64)
          red_add(reinterpret_cast<double*>(P.tally) + slot, __longlong_as_double((long long)val));
        else
          red_add(reinterpret_cast<unsigned long long*>(P.tally) + slot, val);
      }
      return;
    }
    if (emit) {
      const unsigned i = n_st + __popc(m & lanemask_lt());
      S.slot[i] = slot;
      S.val[i] = val;
    }
    n_st += __popc(m);
    if (n_st > kStage - 32) {
      stage_flush(P, S, n_st);
      n_st = 0;
    }
  }
  __device__ __forceinline__ void flush() {
    if (n_st) stage_flush(P, S, n_st);
    n_st = 0;
  }
};

// ------------------------------------------------------------------------------------------ segment scoring
// Scoring apart from the flight (FP32 tracking, tallies of the plain walk): a flown segment is
// written as a record to the warp's segment region, and whenever 32 wait the warp scores 32 of
// them at once, one per lane, for at most kSegRounds rounds; a walk still live then goes back as a
// resumed record, and a finished one comes back for the next tally, if any.  The register-heavy
// walk thus runs outside the flight, and a long walk no longer holds 31 lanes idle.  A resumed
// walk recomputes its crossing distances by the walk's own expressions, so every piece, slot and
// value equals those of an uninterrupted walk.
constexpr unsigned kSegRounds = 3;

struct SegRec {
  float pos[3], u[3], l, t0, s;
  double w;
  int idx[3], it, g, ti;
  bool resumed;
  uint32_t batch;
};

__device__ __forceinline__ void seg_store(uint4* q, unsigned i, const SegRec& r) {
  const unsigned long long wb = (unsigned long long)__double_as_longlong(r.w);
  q[i] = (make_uint4(__float_as_uint(r.pos[0]), __float_as_uint(r.pos[1]), __float_as_uint(r.pos[2]),
                           __float_as_uint(r.u[0])));
  q[kSegCap + i] = (make_uint4(__float_as_uint(r.u[1]), __float_as_uint(r.u[2]), __float_as_uint(r.l),
                                     __float_as_uint(r.t0)));
  q[2 * kSegCap + i] = (make_uint4(__float_as_uint(r.s), r.batch, (uint32_t)wb, (uint32_t)(wb >> 32)));
  q[3 * kSegCap + i] = (
         make_uint4((uint32_t)r.idx[0], (uint32_t)r.idx[1], (uint32_t)r.idx[2],
                    (uint32_t)(r.it + 1) | ((uint32_t)r.g << 17) | ((uint32_t)r.ti << 22) | ((r.resumed ? 1u : 0u) << 24)));
}

__device__ __forceinline__ void seg_load(const uint4* q, unsigned i, SegRec& r) {
  const uint4 a = q[i], b = q[kSegCap + i], c = q[2 * kSegCap + i],
              d = q[3 * kSegCap + i];
  r.pos[0] = __uint_as_float(a.x); r.pos[1] = __uint_as_float(a.y); r.pos[2] = __uint_as_float(a.z);
  r.u[0] = __uint_as_float(a.w); r.u[1] = __uint_as_float(b.x); r.u[2] = __uint_as_float(b.y);
  r.l = __uint_as_float(b.z);
  r.t0 = __uint_as_float(b.w);
  r.s = __uint_as_float(c.x);
  r.w = __longlong_as_double((long long)(((unsigned long long)c.w << 32) | c.z));
  r.idx[0] = (int)d.x; r.idx[1] = (int)d.y; r.idx[2] = (int)d.z;
  r.it = (int)(d.w & 0x1FFFFu) - 1;
  r.g = (int)((d.w >> 17) & 0x1Fu);
  r.ti = (int)((d.w >> 22) & 3u);
  r.resumed = ((d.w >> 24) & 1u) != 0u;
  r.batch = c.y;
}

// the segment a particle is about to fly, for the first tally
__device__ __forceinline__ void seg_push_flight(uint4* q, unsigned i, const Part<float>& p, float l) {
  SegRec r;
  r.pos[0] = p.x; r.pos[1] = p.y; r.pos[2] = p.z;
  r.u[0] = p.ux; r.u[1] = p.uy; r.u[2] = p.uz;
  r.l = l;
  r.t0 = p.time();
  r.s = 0.0f;
  r.w = p.w;
  r.idx[0] = r.idx[1] = r.idx[2] = 0;
  r.it = 0;
  r.g = (int)pk_g(p.pk);
  r.ti = 0;
  r.resumed = false;
  r.batch = p.elem >> 16;
  seg_store(q, i, r);
}

// Scores waiting segments, 32 at a time while 32 wait (or, with `all`, until none is left).
// stripe_off: the CTA's tally stripe.  All 32 lanes call it.
__device__ __forceinline__ void score_segments(const Tab<float>& T, const RunParams& P, uint4* q, unsigned& ns,
                                               bool all, uint64_t stripe_off, const Stage& S, unsigned& pieces) {
  constexpr unsigned kAll = 0xFFFFFFFFu;
  const unsigned lane = threadIdx.x & 31u;
  const char* base = reinterpret_cast<const char*>(T.h);
  const int n_tally = T.h->n_tally;
  while (ns >= 32u || (all && ns > 0u)) {
    const unsigned k = ns < 32u ? ns : 32u;
    const bool have = lane < k;
    SegRec r;
    if (have) seg_load(q, ns - k + lane, r);
    else {
      r.ti = 0;
      r.g = 0;
      r.w = 0.0;
      r.batch = 0u;
      r.t0 = r.l = r.s = 0.0f;
      for (int d = 0; d < 3; ++d) {
        r.pos[d] = 0.0f;
        r.u[d] = 0.0f;
        r.idx[d] = 0;
      }
      r.it = 0;
      r.resumed = true;
    }
    __syncwarp();
    ns -= k;
    const TallyDesc& D = T.h->tally[r.ti];
    const float* e[3] = {reinterpret_cast<const float*>(base + D.o_ex), reinterpret_cast<const float*>(base + D.o_ey),
                         reinterpret_cast<const float*>(base + D.o_ez)};
    const float* et = time_edges<float>(base, D);
    const int n[3] = {D.nx, D.ny, D.nz};
    const int nt = D.nt;
    const float v = T.v[r.g];
    const uint32_t gbase = (uint32_t)(stripe_off + (uint64_t)r.batch * P.row + (uint64_t)D.bin_offset + (uint64_t)r.g * nt);
    const int gstride = T.G * nt;
    float inv[3], sn[3], stn = rinf<float>();
    int step[3];
    bool live = have;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      inv[d] = rdiv(1.0f, r.u[d]);
      step[d] = r.u[d] > 0.0f ? 1 : (r.u[d] < 0.0f ? -1 : 0);
    }
    if (live && !r.resumed) {
      // a new walk: the cells and time bin of the segment's start (as score_segment_warp finds them)
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int i = MCGB_BIN_GUESS ? bin_find(e[d], n[d], r.pos[d], D.gkind[d], D.ga[d], D.gb[d])
                                     : bin_search(e[d], n[d], r.pos[d]);
        r.idx[d] = i;
        if (step[d] > 0) {
          if (i >= n[d]) live = false;
          sn[d] = (i >= n[d]) ? rinf<float>() : (e[d][i + 1] - r.pos[d]) * inv[d];
        } else if (step[d] < 0) {
          if (i < 0) live = false;
          sn[d] = (i < 0) ? rinf<float>() : (e[d][i] - r.pos[d]) * inv[d];
        } else {
          sn[d] = rinf<float>();
          if (i < 0 || i >= n[d]) live = false;
        }
      }
      r.it = MCGB_BIN_GUESS ? bin_find(et, nt, r.t0, D.gkind[3], D.ga[3], D.gb[3]) : bin_search(et, nt, r.t0);
      if (r.it >= nt) live = false;
      else stn = (et[r.it + 1] - r.t0) * v;
    } else if (live) {
#pragma unroll
      for (int d = 0; d < 3; ++d)
        sn[d] = step[d] > 0 ? (e[d][r.idx[d] + 1] - r.pos[d]) * inv[d]
                            : (step[d] < 0 ? (e[d][r.idx[d]] - r.pos[d]) * inv[d] : rinf<float>());
      stn = (et[r.it + 1] - r.t0) * v;
    }
    ScoreSink<float> sink(P, S, pieces, r.w);
    for (unsigned rounds = 0; rounds < kSegRounds && __any_sync(kAll, live); ++rounds) {
      bool emit = false;
      uint32_t slot = 0;
      float len = 0.0f;
      if (live) {
        const float nxt = fmin(fmin(fmin(sn[0], sn[1]), fmin(sn[2], stn)), r.l);
        emit = nxt > r.s && r.idx[0] >= 0 && r.idx[0] < n[0] && r.idx[1] >= 0 && r.idx[1] < n[1] && r.idx[2] >= 0 &&
               r.idx[2] < n[2] && r.it >= 0;
        slot = gbase + (uint32_t)(((r.idx[2] * n[1] + r.idx[1]) * n[0] + r.idx[0]) * gstride + r.it);
        len = nxt - r.s;
        bool alive = nxt < r.l;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const bool st = sn[d] <= nxt;
          const int ni = r.idx[d] + (st ? step[d] : 0);
          const int ei = min(max(ni + (step[d] > 0 ? 1 : 0), 0), n[d]);
          const float nsn = (e[d][ei] - r.pos[d]) * inv[d];
          alive = alive && !(st && (ni < 0 || ni >= n[d]));
          r.idx[d] = ni;
          sn[d] = st ? nsn : sn[d];
        }
        {
          const bool st = stn <= nxt;
          const int ni = r.it + (st ? 1 : 0);
          const float nstn = (et[min(ni + 1, nt)] - r.t0) * v;
          alive = alive && ni < nt;
          r.it = ni;
          stn = st ? nstn : stn;
        }
        live = alive;
        r.s = nxt;
      }
      sink.add(emit, slot, len);
    }
    sink.flush();
    // back to the region: the rest of a live walk, or the segment again for the next tally
    const bool next_tally = have && !live && r.ti + 1 < n_tally;
    const bool put = live || next_tally;
    if (next_tally) {
      r.ti += 1;
      r.resumed = false;
      r.s = 0.0f;
    } else {
      r.resumed = true;
    }
    const unsigned m = __ballot_sync(kAll, put);
    if (put) seg_store(q, ns + __popc(m & lanemask_lt()), r);
    ns += __popc(m);
  }
}

// Track-length estimator over the segment of length l from the particle's position: score
// w * piece length into every (mesh cell, time bin) the segment passes through.  Crossing
// distances are measured from the segment start, so rounding does not accumulate along the walk.
// The walk runs in warp-uniform rounds; pieces go to the warp's staging buffer, which is flushed
// with converged lanes whenever it could overflow and at the end.  Called by all 32 lanes;
// `active` lanes have a segment.
//
// Plain walk: every round each walking lane emits one piece, the part of its segment up to the
// next crossing of a mesh plane or time edge.
//
// Range walk (TallyDesc::range, a time axis much finer than the spatial mesh, so that a flight
// crosses many more time edges than planes): every round each lane takes one mesh cell.  Its
// sub-segment [s, e) there spans time bins first..last, found by binary search over the edge
// distances D_k = (t_k - t0) v.  A bin strictly inside that span is crossed in full, and the
// track length of a full bin k is the constant v (t_{k+1} - t_k): the lane scores the two end bins
// as pieces and the run of full bins first+1 .. last-1 as two difference marks, +w at first+1 and
// -w at last, in the tally's difference slots.  A reconstruction pass after the run turns the
// running sum of the marks into w v (t_{k+1} - t_k) per bin.  A lane thus makes at most four
// updates per cell, however many time bins its flight crosses.
//
// RANGE = false compiles only the plain walk, which keeps the kernel's register footprint down.
template <typename R, bool RANGE>
__device__ void score_segment_warp(const Tab<R>& T, const RunParams& P, const Part<R>& p, R l,
                                   uint64_t batch_base, bool active, const Stage& S, unsigned& pieces) {
  constexpr unsigned kAll = 0xFFFFFFFFu;
  const unsigned lt = lanemask_lt();
  const int g = (int)pk_g(p.pk);
  const R v = active ? T.v[g] : R(1);
  const char* base = reinterpret_cast<const char*>(T.h);
  const R t0 = active ? p.time() : R(0);
  const double w = active ? p.w : 0.0;
  const float wscale = sizeof(R) == 4 ? weight_to_float(w) * P.fixed_scale_f : 0.0f;
  const bool fp32_fixed = sizeof(R) == 4 && !P.tally_fp64;
  unsigned n_st = 0;
  const bool direct = !P.aggregate;  // warp-uniform
  // stages one value per lane (those with emit), flushing when the buffer could overflow; without
  // warp aggregation the staging buys nothing, and each lane adds its value at once (fire-and-
  // forget atomics; integer sums do not depend on their order)
  auto stage_bits = [&](bool emit, uint32_t slot, unsigned long long val) {
    const unsigned m = __ballot_sync(kAll, emit);
    if (direct) {
      pieces += __popc(m);
      if (emit && in_range(P, slot, (uint64_t)P.tally_stripes * P.stripe_stride)) {
        if (P.tally_fp64)
          red_add(reinterpret_cast<double*>(P.tally) + slot, __longlong_as_double((long long)val));
        else
          red_add(reinterpret_cast<unsigned long long*>(P.tally) + slot, val);
      }
      return;
    }
    if (emit) {
      const unsigned i = n_st + __popc(m & lt);
      S.slot[i] = slot;
      S.val[i] = val;
    }
    n_st += __popc(m);
    pieces += __popc(m);  // warp-uniform count, added to the counters at the end
    if (n_st > kStage - 32) {
      stage_flush(P, S, n_st);
      n_st = 0;
    }
  };
  // the score of a piece of length len (or, with len = +-1, a difference mark of +-w)
  auto score_val = [&](bool emit, R len) -> unsigned long long {
    if (!emit) return 0ull;
    if (fp32_fixed) {
      const long long q = float_to_fixed(wscale * fabsf((float)len));
      return (unsigned long long)(len < R(0) ? -q : q);
    }
    return score_bits_fp64(P, w, (double)len);
  };
  auto stage = [&](bool emit, uint32_t slot, R len) { stage_bits(emit, slot, score_val(emit, len)); };
  for (int ti = 0; ti < T.h->n_tally; ++ti) {
    const TallyDesc& D = T.h->tally[ti];
    const R* e[3] = {reinterpret_cast<const R*>(base + D.o_ex), reinterpret_cast<const R*>(base + D.o_ey),
                     reinterpret_cast<const R*>(base + D.o_ez)};
    const R* et = time_edges<R>(base, D);
    const int n[3] = {D.nx, D.ny, D.nz};
    const int nt = D.nt;
    const bool crossing = D.est == MC_EST_TIME_CROSSING;
    if (crossing && !(RANGE && D.range)) {
      // Time-crossing estimator: at every time point t_j with t0 <= t_j < t0 + l / v the particle
      // scores its weight into the mesh cell it occupies at t_j (the readback multiplies by v_g).
      // One point per lane per warp-uniform round.
      bool live = active;
      int j = 0;
      R dj = R(0);  // distance along the flight to point j
      if (live) {
        int lo = 0, hi = nt + 1;  // first point at or after the flight's start
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (et[mid] < t0) lo = mid + 1;
          else hi = mid;
        }
        j = lo;
        if (j > nt) live = false;
        else {
          dj = (et[j] - t0) * v;
          live = dj < l;
        }
      }
      const uint32_t cb = (uint32_t)(batch_base + (uint64_t)D.bin_offset + (uint64_t)g * D.nval);
      const int cs = T.G * D.nval;
      while (__any_sync(kAll, live)) {
        bool emit = false;
        uint32_t slot = 0;
        if (live) {
          const R sd = dj > R(0) ? dj : R(0);
          const int ix = bin_search(e[0], n[0], p.x + sd * p.ux), iy = bin_search(e[1], n[1], p.y + sd * p.uy),
                    iz = bin_search(e[2], n[2], p.z + sd * p.uz);
          if (ix >= 0 && ix < n[0] && iy >= 0 && iy < n[1] && iz >= 0 && iz < n[2]) {
            emit = true;
            slot = cb + (uint32_t)(((iz * n[1] + iy) * n[0] + ix) * cs + j);
          }
          ++j;
          if (j > nt) live = false;
          else {
            dj = (et[j] - t0) * v;
            live = dj < l;
          }
        }
        stage(emit, slot, R(1));
      }
      continue;
    }
    R pos[3], u[3], sn[3], inv[3], s = R(0), stn = rinf<R>();  // stn: distance to time edge it+1
    int idx[3], step[3], it = 0;
    bool live = active;
    if (live) {
      pos[0] = p.x; pos[1] = p.y; pos[2] = p.z;
      u[0] = p.ux; u[1] = p.uy; u[2] = p.uz;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const int i = bin_search(e[d], n[d], pos[d]);
        idx[d] = i;
        inv[d] = rdiv(R(1), u[d]);
        if (u[d] > R(0)) {
          step[d] = 1;
          if (i >= n[d]) live = false;
          sn[d] = (i >= n[d]) ? rinf<R>() : (e[d][i + 1] - pos[d]) * inv[d];
        } else if (u[d] < R(0)) {
          step[d] = -1;
          if (i < 0) live = false;
          sn[d] = (i < 0) ? rinf<R>() : (e[d][i] - pos[d]) * inv[d];
        } else {
          step[d] = 0;
          sn[d] = rinf<R>();
          if (i < 0 || i >= n[d]) live = false;
        }
      }
      if (!crossing) {
        it = bin_search(et, nt, t0);  // -1 before the first edge; then D_it <= s < D_it+1
        if (it >= nt) live = false;
        else stn = (et[it + 1] - t0) * v;
      }
    }
    if (crossing) {
      // Time-crossing range walk: one mesh cell per lane per round.  The points the flight spans
      // while in that cell, D_j in [s, end), are a run jn .. jb that all score w into the cell: one
      // direct score for a single point, else two difference marks (+w at jn, -w at jb + 1) that
      // the reconstruction turns into w at every point of the run.
      int jn = 0;  // the next point: first j with D_j >= s
      if (live) {
        int lo = 0, hi = nt + 1;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (et[mid] < t0) lo = mid + 1;
          else hi = mid;
        }
        jn = lo;
        if (jn > nt) live = false;
      }
      const uint32_t cb = (uint32_t)(batch_base + (uint64_t)D.bin_offset + (uint64_t)g * D.nval);
      const int cs = T.G * D.nval;
      const uint32_t db = (uint32_t)(batch_base + (uint64_t)T.h->total_bins + (uint64_t)D.diff_offset +
                                     (uint64_t)g * D.ndiff);
      const int dstride = T.G * D.ndiff;
      while (__any_sync(kAll, live)) {
        R end = s;
        int ja = 0, jb = -1;
        uint32_t cell = 0;
        if (live) {
          end = fmin(fmin(fmin(sn[0], sn[1]), sn[2]), l);
          int lo = jn - 1, hi = nt;  // the last point with D_j < end (jn - 1: none)
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((et[mid] - t0) * v < end) lo = mid;
            else hi = mid - 1;
          }
          if (end > s && lo >= jn && idx[0] >= 0 && idx[0] < n[0] && idx[1] >= 0 && idx[1] < n[1] && idx[2] >= 0 &&
              idx[2] < n[2]) {
            ja = jn;
            jb = lo;
            cell = (uint32_t)((idx[2] * n[1] + idx[1]) * n[0] + idx[0]);
          }
          jn = lo + 1;
        }
        stage(jb == ja, cb + cell * (uint32_t)cs + (uint32_t)ja, R(1));
        if (__any_sync(kAll, jb > ja)) {
          const bool run = jb > ja;
          const uint32_t dc = db + cell * (uint32_t)dstride;
          stage(run, dc + (uint32_t)ja, R(1));
          stage(run, dc + (uint32_t)(jb + 1), R(-1));
        }
        if (live) {
          if (end >= l || jn > nt) {
            live = false;  // the flight or the time points ended
          } else {
#pragma unroll
            for (int d = 0; d < 3; ++d) {
              if (sn[d] <= end) {
                idx[d] += step[d];
                if (idx[d] < 0 || idx[d] >= n[d]) live = false;  // left the mesh along this axis
                else sn[d] = (e[d][idx[d] + (step[d] > 0 ? 1 : 0)] - pos[d]) * inv[d];
              }
            }
          }
          s = end;
        }
      }
      continue;
    }
    const uint32_t gbase = (uint32_t)(batch_base + (uint64_t)D.bin_offset + (uint64_t)g * nt);
    const int gstride = T.G * nt;
    if (!RANGE || !D.range) {
      while (__any_sync(kAll, live)) {
        bool emit = false;
        uint32_t slot = 0;
        R len = R(0);
        if (live) {
          const R nxt = fmin(fmin(fmin(sn[0], sn[1]), fmin(sn[2], stn)), l);
          emit = nxt > s && idx[0] >= 0 && idx[0] < n[0] && idx[1] >= 0 && idx[1] < n[1] && idx[2] >= 0 &&
                 idx[2] < n[2] && it >= 0;
          slot = gbase + (uint32_t)(((idx[2] * n[1] + idx[1]) * n[0] + idx[0]) * gstride + it);
          len = nxt - s;
          // every axis (and the time axis) whose crossing is at nxt steps, without branches: the next
          // crossing distance is computed for every axis (edge index clamped to the edge list) and
          // kept only where the axis stepped; an axis stepping out of the mesh ends the walk
          bool alive = nxt < l;
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const bool st = sn[d] <= nxt;
            const int ni = idx[d] + (st ? step[d] : 0);
            const int ei = min(max(ni + (step[d] > 0 ? 1 : 0), 0), n[d]);
            const R nsn = (e[d][ei] - pos[d]) * inv[d];
            alive = alive && !(st && (ni < 0 || ni >= n[d]));
            idx[d] = ni;
            sn[d] = st ? nsn : sn[d];
          }
          {
            const bool st = stn <= nxt;
            const int ni = it + (st ? 1 : 0);
            const R nstn = (et[min(ni + 1, nt)] - t0) * v;
            alive = alive && ni < nt;
            it = ni;
            stn = st ? nstn : stn;
          }
          live = alive;
          s = nxt;
        }
        stage(emit, slot, len);
      }
      continue;
    }
    // difference slots of this (group, cell): nt + 1 marks per (cell, group) after the batch row's
    // bins; mark k belongs to bin k
    const uint32_t dbase = (uint32_t)(batch_base + (uint64_t)T.h->total_bins + (uint64_t)D.diff_offset +
                                      (uint64_t)g * D.ndiff);
    const int dstride = T.G * D.ndiff;
    while (__any_sync(kAll, live)) {
      // this lane's sub-segment [s, end) in mesh cell idx, and the last time edge klt before end:
      // it spans time bins max(it, 0) .. min(klt, nt - 1)
      R end = s;
      int klt = it, first = 0, last = -1;
      uint32_t cell = 0;
      if (live) {
        end = fmin(fmin(fmin(sn[0], sn[1]), sn[2]), l);
        if (stn < end) {
          int lo = it + 1, hi = nt;
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if ((et[mid] - t0) * v < end) lo = mid;
            else hi = mid - 1;
          }
          klt = lo;
        }
        if (end > s && idx[0] >= 0 && idx[0] < n[0] && idx[1] >= 0 && idx[1] < n[1] && idx[2] >= 0 &&
            idx[2] < n[2]) {
          first = it > 0 ? it : 0;
          last = klt < nt - 1 ? klt : nt - 1;
          cell = (uint32_t)((idx[2] * n[1] + idx[1]) * n[0] + idx[0]);
        }
      }
      const bool any = last >= first;
      // piece in bin `first`: from s (or its lower edge) to its upper edge (or end)
      {
        const R lo = first == it ? s : (et[first] - t0) * v;
        const R hi = first < klt ? (et[first + 1] - t0) * v : end;
        stage(any && hi > lo, gbase + cell * (uint32_t)gstride + (uint32_t)first, hi - lo);
      }
      if (__any_sync(kAll, last > first)) {
        const bool two = last > first;
        // piece in bin `last`, from its lower edge to end (or its upper edge, past the time mesh)
        const R lo = (et[last] - t0) * v;
        const R hi = last < klt ? (et[last + 1] - t0) * v : end;
        stage(two && hi > lo, gbase + cell * (uint32_t)gstride + (uint32_t)last, hi - lo);
        if (__any_sync(kAll, last > first + 1)) {
          const bool full = last > first + 1;
          const uint32_t db = dbase + cell * (uint32_t)dstride;
          stage(full, db + (uint32_t)(first + 1), R(1));
          stage(full, db + (uint32_t)last, R(-1));
        }
      }
      // advance along the walk (lane-local)
      if (live) {
        if (klt >= nt) {
          live = false;  // the time mesh ended inside this sub-segment
        } else {
          const R dn = klt == it ? stn : (et[klt + 1] - t0) * v;  // distance to edge klt+1
          if (dn <= end) {
            it = klt + 1;
            if (it >= nt) live = false;
            else stn = (et[it + 1] - t0) * v;
          } else if (klt != it) {
            it = klt;
            stn = dn;
          }
        }
        if (end >= l) {
          live = false;
        } else if (live) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            if (sn[d] <= end) {
              idx[d] += step[d];
              if (idx[d] < 0 || idx[d] >= n[d]) live = false;  // left the mesh along this axis
              else sn[d] = (e[d][idx[d] + (step[d] > 0 ? 1 : 0)] - pos[d]) * inv[d];
            }
          }
        }
        s = end;
      }
    }
  }
  if (n_st) stage_flush(P, S, n_st);
}

// ------------------------------------------------------------------------------------------ sampling
template <typename R>
__device__ __forceinline__ int sample_cdf(const R* cdf, int n, R u) {
  for (int i = 0; i < n; ++i)
    if (u < cdf[i]) return i;
  return n - 1;
}

template <typename R>
__device__ __forceinline__ void iso_dir(R mu, R uphi, R& ux, R& uy, R& uz) {
  R s, c;
  sincos2pi(uphi, &s, &c);
  const R sn = rsqrt_(fmax(R(0), R(1) - mu * mu));
  ux = mu;
  uy = sn * c;
  uz = sn * s;
}

}  // namespace mcgb
