// Pixel kernels: the hot loop of the method.
//
// For every (source, image patch, pixel tile) work item, one warp stages the
// pair's component record in shared memory and each lane walks its pixels:
//   * renders the source's galaxy and star profile densities with their
//     first and second derivatives in the image's natural coordinates
//     (centre mu, shape G = A Sigma_s A^T, profile weight rho) -- Sec. 2.2.3;
//   * forms E = bgE + E_s and V = bgV + V_s (Eqs. conditional, vareq) and the
//     delta-method pixel term -E + x (log E - V / (2 E^2)) (Eq. eq:log_p_last,
//     Sec. 4.2.2) with its partials;
//   * accumulates the value, the gradient and the Hessian over the 10
//     per-image natural coordinates w = (cE0, cE1, cM0, cM1, mu, G, rho).
// The warp reduces its 64 sums with shuffles and writes them to the item's
// slot; the epilogue adds a pair's items (compensated FP32, the value sums
// in FP64) and chains them to the 27 coordinates.
//
// Derivatives of a Gaussian component with respect to its covariance come
// from the heat equation (d phi / dC_ab = 1/2 d^2 phi / dmu_a dmu_b), so the
// kernel only needs the Hermite polynomials of orders 0..4 in y = P (p - mu).
#include <math.h>

#include "device_once.h"
#include "internal.cuh"
#include "setup.cuh"

namespace celeste {

constexpr float kHalfLog2e = 0.72134752044448170368f;   // log2(e) / 2

// ---- staged records
// Every pixel kernel stages the (source, image) record of its work item in
// the warp's shared memory, built from the global record (8 floats per
// component: mx, my, P11, P12, P22, lw, tau) in one of two layouts:
//   value layout:  header | origins | star {A11, A12, A22, lw}
//                                   | per PSF component k: galaxy pairs, then singles
//   derivs layout: header | origins | star {A, lw | P, 0}
//                                   | per PSF component k: galaxy pairs, then singles
// A galaxy component has 16 values {A, lw | -P11, -P12, -P22, tau |
// -2 P12, -2 P11^2, -2 P22^2, -2 P12^2 | -4 P12, -2 P12 P11, -2 P12 P22, 0}:
// the signs are chosen so that no formula below negates an operand.  The components of PSF
// component k come in pairs (exponential j, de Vaucouleurs j) for
// j < min(n_exp, n_dev), their values interleaved (exponential in the even
// slots), so that one packed two-wide FP32 instruction (ffma2, which rounds
// each half as fmaf does) evaluates both; the components without a partner
// follow with their 16 values in a row.
// A = -log2(e)/2 (P11, 2 P12, P22) are the coefficients of the exponent's
// quadratic form: log2 phi = lw + A11 dx^2 + A12 dx dy + A22 dy^2.  Every
// component convolved with PSF component k has that component's mean (the
// source centre plus the PSF offset), so a kernel forms the pixel's offset
// and its products once per k from the "origins".  Both layouts evaluate
// phi with the same instructions: a value-only kernel and the derivative
// kernel give bit-identical densities for the same record.
constexpr int kOrgF = 8;                                   // (mx, my) per k, padded
constexpr int kValF = 4;
constexpr int kStarF = 8;
constexpr int kGalF = 16;
constexpr int kCompBase = kHdr + kOrgF;
constexpr int kValRecF = kCompBase + kMaxComp * kValF;
constexpr int kDerivRecF = kCompBase + kPsf * kStarF + kPsf * 2 * kMaxProf * kGalF;
static_assert(2 * kPsf <= kOrgF && kValRecF % 4 == 0 && kDerivRecF % 4 == 0, "staged layout");

__device__ __forceinline__ float4 quad_coeffs(float p11, float p12, float p22, float lw) {
  return make_float4(-kHalfLog2e * p11, (-2.f * kHalfLog2e) * p12, -kHalfLog2e * p22, lw);
}

// Stages the record at src (global) into dst (the warp's shared memory);
// n_comp = kPsf (1 + n_exp + n_dev) components in the global order (stars,
// then per PSF component the exponential and de Vaucouleurs components).
template <bool kDerivs>
__device__ __forceinline__ void stage_record(float* __restrict__ dst, const float* __restrict__ src,
                                             int n_comp, int lane, int n_exp = 0) {
  const float4* s4 = reinterpret_cast<const float4*>(src);
  float4* d4 = reinterpret_cast<float4*>(dst);
  if (lane < kHdr / 4) d4[lane] = s4[lane];
  if (lane < kPsf)
    *reinterpret_cast<float2*>(dst + kHdr + 2 * lane) =
        *reinterpret_cast<const float2*>(src + kHdr + lane * kCompF);
  for (int ci = lane; ci < n_comp; ci += 32) {
    const float4 a = s4[kHdr / 4 + 2 * ci];
    const float4 b = s4[kHdr / 4 + 2 * ci + 1];
    const float p11 = a.z, p12 = a.w, p22 = b.x;
    const float4 q = quad_coeffs(p11, p12, p22, b.y);
    if (!kDerivs) {
      if (ci < kPsf) {
        d4[kCompBase / 4 + ci] = q;
      } else {
        // galaxy: pairs (exponential j, de Vaucouleurs j) interleaved, then
        // the components without a partner
        const int per = (n_comp - kPsf) / kPsf;
        const int g = ci - kPsf, k = g / per, jj = g - k * per;
        const int nb = n_exp < per - n_exp ? n_exp : per - n_exp;
        const bool dev = jj >= n_exp;
        const int j = dev ? jj - n_exp : jj;
        float* base = dst + kCompBase + (kPsf + k * per) * kValF;
        if (j < nb) {
          float* o = base + j * 2 * kValF + (dev ? 1 : 0);
          o[0] = q.x;
          o[2] = q.y;
          o[4] = q.z;
          o[6] = q.w;
        } else {
          const int single = dev ? (n_exp - nb) + (j - nb) : j - nb;
          *reinterpret_cast<float4*>(base + nb * 2 * kValF + single * kValF) = q;
        }
      }
    } else if (ci < kPsf) {
      float4* o = reinterpret_cast<float4*>(dst + kCompBase + ci * kStarF);
      o[0] = q;
      o[1] = make_float4(p11, p12, p22, 0.f);
    } else {
      // galaxy component: PSF component k, index j of its profile
      const int per = (n_comp - kPsf) / kPsf;
      const int g = ci - kPsf, k = g / per, jj = g - k * per;
      const int ne = n_exp;
      const int nb = ne < per - ne ? ne : per - ne;
      const bool dev = jj >= ne;
      const int j = dev ? jj - ne : jj;
      const float vals[kGalF] = {q.x, q.y, q.z, q.w, -p11, -p12, -p22, b.z,
                                 -2.f * p12, -2.f * p11 * p11, -2.f * p22 * p22, -2.f * p12 * p12,
                                 -4.f * p12, (-2.f * p12) * p11, (-2.f * p12) * p22, 0.f};
      float* base = dst + kCompBase + kPsf * kStarF + k * per * kGalF;
      if (j < nb) {
        float* o = base + j * 2 * kGalF + (dev ? 1 : 0);
#pragma unroll
        for (int e = 0; e < kGalF; ++e) o[2 * e] = vals[e];
      } else {
        const int single = dev ? (ne - nb) + (j - nb) : j - nb;
        float4* o = reinterpret_cast<float4*>(base + nb * 2 * kGalF + single * kGalF);
#pragma unroll
        for (int e = 0; e < kGalF / 4; ++e)
          o[e] = make_float4(vals[4 * e], vals[4 * e + 1], vals[4 * e + 2], vals[4 * e + 3]);
      }
    }
  }
}

// A pixel's offset from PSF component k's mean, and its products.
struct Offset {
  float dx, dy, xx, xy, yy;
};
__device__ __forceinline__ float2 pixel_delta(const float* __restrict__ rec, int k, float px,
                                              float py) {
  const float2 m = *reinterpret_cast<const float2*>(rec + kHdr + 2 * k);
  return make_float2(px - m.x, py - m.y);
}
__device__ __forceinline__ Offset make_offset(float2 d) {
  return Offset{d.x, d.y, d.x * d.x, d.x * d.y, d.y * d.y};
}
// Work units of a launch for one warp.  Warp w starts with unit w; with a
// queue q ([0]: units handed out beyond the first per warp, [1]: warps done;
// zero between launches) a warp then takes the next free unit whenever it
// finishes one, asking for it while it works on the current one, so every
// warp stays busy until the last unit; the last warp of the launch to finish
// resets the queue.  Without one (q null) units are dealt out by grid
// stride.  Every warp of the launch must reach done().
struct WarpQueue {
  int32_t* q;
  int it, next, stride;
  __device__ __forceinline__ WarpQueue(int32_t* queue) : q(queue), next(0) {
    stride = gridDim.x * (blockDim.x >> 5);
    it = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  }
  // at the top of every unit, before any continue
  __device__ __forceinline__ void ask(int lane) {
    if (q && lane == 0) next = stride + atomicAdd(q, 1);
  }
  __device__ __forceinline__ void advance() {
    it = q ? __shfl_sync(0xffffffffu, next, 0) : it + stride;
  }
  __device__ __forceinline__ void done(int lane) {
    if (q && lane == 0) {
      __threadfence();
      if (atomicAdd(q + 1, 1) == stride - 1) {
        q[0] = 0;
        q[1] = 0;
      }
    }
  }
};

// A lane's pixels q0, q0 + step, q0 + 2 step, ... (step 32 unless given) of
// a row-major patch of width w as (column, row), without a division per
// pixel: a step is ay rows and ax columns, plus one row when the column
// passes w.
struct PixelWalk {
  int qx, qy, ax, ay;
  __device__ __forceinline__ PixelWalk(int q0, int w, int step = 32) {
    qy = q0 / w;
    qx = q0 - qy * w;
    ay = step / w;
    ax = step - ay * w;
  }
  __device__ __forceinline__ void next(int w) {
    qx += ax;
    qy += ay;
    if (qx >= w) {
      qx -= w;
      ++qy;
    }
  }
};

// Density (weight and normaliser included) of a component with coefficients q.
__device__ __forceinline__ float gauss_density(const float4 q, const Offset& o) {
  return exp2f(fmaf(q.x, o.xx, fmaf(q.y, o.xy, fmaf(q.z, o.yy, q.w))));
}

// Sums over the components of one galaxy profile (weights without rho):
// S*: derivatives in mu; T2: tau-weighted second order (-> dG);
// T3: tau-weighted third order (-> d mu dG); T4: tau^2 fourth order (-> dG dG).
// The odd orders (s1*, t3*) are accumulated with the opposite sign: the
// kernels form z = -y = (-P) (p - mu) from the staged -P, and the Hermite
// polynomials of odd order change sign with y.
struct GalSums {
  float s0, s1x, s1y, s2xx, s2xy, s2yy;
  float t2xx, t2xy, t2yy;
  float t3a, t3b, t3c, t3d;            // 111, 112, 122, 222
  float t4a, t4b, t4c, t4d, t4e;       // 1111, 1112, 1122, 1222, 2222
};

// One galaxy component of the derivs layout (16 staged values).
__device__ __forceinline__ void gal_accumulate(const float* __restrict__ c, const Offset& o,
                                               GalSums& g) {
  const float4 q = *reinterpret_cast<const float4*>(c);
  const float4 pp = *reinterpret_cast<const float4*>(c + 4);
  const float4 hc = *reinterpret_cast<const float4*>(c + 8);
  const float4 hd = *reinterpret_cast<const float4*>(c + 12);
  const float m4P12 = hd.x, c4b = hd.y, c4d = hd.z;
  const float nP11 = pp.x, nP12 = pp.y, nP22 = pp.z, tau = pp.w, m2P12 = hc.x;
  const float z1 = fmaf(nP11, o.dx, nP12 * o.dy);       // -y1
  const float z2 = fmaf(nP12, o.dx, nP22 * o.dy);       // -y2
  const float phi = gauss_density(q, o);
  const float h11 = fmaf(z1, z1, nP11);                 // y y^T - P
  const float h12 = fmaf(z1, z2, nP12);
  const float h22 = fmaf(z2, z2, nP22);
  const float pt = phi * tau;
  const float pt2 = pt * tau;
  g.s0 += phi;
  g.s1x = fmaf(phi, z1, g.s1x);
  g.s1y = fmaf(phi, z2, g.s1y);
  g.s2xx = fmaf(phi, h11, g.s2xx);
  g.s2xy = fmaf(phi, h12, g.s2xy);
  g.s2yy = fmaf(phi, h22, g.s2yy);
  g.t2xx = fmaf(pt, h11, g.t2xx);
  g.t2xy = fmaf(pt, h12, g.t2xy);
  g.t2yy = fmaf(pt, h22, g.t2yy);
  // third order: y_a y_b y_c - (P_ab y_c + P_ac y_b + P_bc y_a)
  const float a1 = fmaf(2.f, nP11, h11), a2 = fmaf(2.f, nP22, h22);
  const float pz1 = pt * z1, pz2 = pt * z2;
  g.t3a = fmaf(pz1, a1, g.t3a);
  g.t3b = fmaf(pz2, h11, fmaf(m2P12, pz1, g.t3b));
  g.t3c = fmaf(pz1, h22, fmaf(m2P12, pz2, g.t3c));
  g.t3d = fmaf(pz2, a2, g.t3d);
  // fourth order, written with h = y y^T - P (y1^2 = h11 + P11, y2^2 =
  // h22 + P22: the -2 P12 P terms are staged)
  g.t4a = fmaf(pt2, fmaf(h11, fmaf(4.f, nP11, h11), hc.y), g.t4a);
  g.t4b = fmaf(pt2, fmaf(h12, a1, fmaf(m2P12, h11, c4b)), g.t4b);
  g.t4c = fmaf(pt2, fmaf(h11, h22, fmaf(h12, m4P12, hc.w)), g.t4c);
  g.t4d = fmaf(pt2, fmaf(h12, a2, fmaf(m2P12, h22, c4d)), g.t4d);
  g.t4e = fmaf(pt2, fmaf(h22, fmaf(4.f, nP22, h22), hc.z), g.t4e);
}

// ---- packed pairs (exponential j, de Vaucouleurs j) ------------------------
// ffma2 / fmul2 / fadd2 round each half exactly as fmaf / * / + do, so the
// packed sums equal, bit for bit, the ones the scalar code forms.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// A pixel's offset products, duplicated in both halves.
struct Offset2 {
  float2 dx, dy, xx, xy, yy;
};
__device__ __forceinline__ Offset2 dup_offset(const Offset& o) {
  return Offset2{f2(o.dx), f2(o.dy), f2(o.xx), f2(o.xy), f2(o.yy)};
}

// The sums of GalSums for both profiles: .x exponential, .y de Vaucouleurs.
struct GalSums2 {
  float2 s0, s1x, s1y, s2xx, s2xy, s2yy;
  float2 t2xx, t2xy, t2yy;
  float2 t3a, t3b, t3c, t3d;
  float2 t4a, t4b, t4c, t4d, t4e;
};

// gal_accumulate on a staged pair (32 floats, exponential in the even slots).
__device__ __forceinline__ void gal_accumulate2(const float* __restrict__ c, const Offset2& o,
                                                GalSums2& g) {
  const float4 qa = *reinterpret_cast<const float4*>(c);
  const float4 qb = *reinterpret_cast<const float4*>(c + 4);
  const float4 pa = *reinterpret_cast<const float4*>(c + 8);
  const float4 pb = *reinterpret_cast<const float4*>(c + 12);
  const float4 ha = *reinterpret_cast<const float4*>(c + 16);
  const float4 hb = *reinterpret_cast<const float4*>(c + 20);
  const float4 hq = *reinterpret_cast<const float4*>(c + 24);
  const float2 c4d = *reinterpret_cast<const float2*>(c + 28);
  const float2 m4P12 = make_float2(hq.x, hq.y), c4b = make_float2(hq.z, hq.w);
  const float2 A11 = make_float2(qa.x, qa.y), A12 = make_float2(qa.z, qa.w);
  const float2 A22 = make_float2(qb.x, qb.y), lw = make_float2(qb.z, qb.w);
  const float2 nP11 = make_float2(pa.x, pa.y), nP12 = make_float2(pa.z, pa.w);
  const float2 nP22 = make_float2(pb.x, pb.y), tau = make_float2(pb.z, pb.w);
  const float2 m2P12 = make_float2(ha.x, ha.y), c4a = make_float2(ha.z, ha.w);
  const float2 c4e = make_float2(hb.x, hb.y), c4c = make_float2(hb.z, hb.w);
  const float2 two = f2(2.f), four = f2(4.f);
  const float2 z1 = fma2(nP11, o.dx, mul2(nP12, o.dy));
  const float2 z2 = fma2(nP12, o.dx, mul2(nP22, o.dy));
  const float2 arg = fma2(A11, o.xx, fma2(A12, o.xy, fma2(A22, o.yy, lw)));
  const float2 phi = make_float2(exp2f(arg.x), exp2f(arg.y));
  const float2 h11 = fma2(z1, z1, nP11);
  const float2 h12 = fma2(z1, z2, nP12);
  const float2 h22 = fma2(z2, z2, nP22);
  const float2 pt = mul2(phi, tau);
  const float2 pt2 = mul2(pt, tau);
  g.s0 = add2(g.s0, phi);
  g.s1x = fma2(phi, z1, g.s1x);
  g.s1y = fma2(phi, z2, g.s1y);
  g.s2xx = fma2(phi, h11, g.s2xx);
  g.s2xy = fma2(phi, h12, g.s2xy);
  g.s2yy = fma2(phi, h22, g.s2yy);
  g.t2xx = fma2(pt, h11, g.t2xx);
  g.t2xy = fma2(pt, h12, g.t2xy);
  g.t2yy = fma2(pt, h22, g.t2yy);
  const float2 a1 = fma2(two, nP11, h11), a2 = fma2(two, nP22, h22);
  const float2 pz1 = mul2(pt, z1), pz2 = mul2(pt, z2);
  g.t3a = fma2(pz1, a1, g.t3a);
  g.t3b = fma2(pz2, h11, fma2(m2P12, pz1, g.t3b));
  g.t3c = fma2(pz1, h22, fma2(m2P12, pz2, g.t3c));
  g.t3d = fma2(pz2, a2, g.t3d);
  g.t4a = fma2(pt2, fma2(h11, fma2(four, nP11, h11), c4a), g.t4a);
  g.t4b = fma2(pt2, fma2(h12, a1, fma2(m2P12, h11, c4b)), g.t4b);
  g.t4c = fma2(pt2, fma2(h11, h22, fma2(h12, m4P12, c4c)), g.t4c);
  g.t4d = fma2(pt2, fma2(h12, a2, fma2(m2P12, h22, c4d)), g.t4d);
  g.t4e = fma2(pt2, fma2(h22, fma2(four, nP22, h22), c4e), g.t4e);
}

// A component without a partner: gal_accumulate into half L of g.
template <int L>
__device__ __forceinline__ void gal_single(const float* __restrict__ c, const Offset& o,
                                           GalSums2& g) {
  GalSums h;
#define GET(f) h.f = L ? g.f.y : g.f.x;
#define PUT(f) (L ? g.f.y : g.f.x) = h.f;
#define ALL(M) M(s0) M(s1x) M(s1y) M(s2xx) M(s2xy) M(s2yy) M(t2xx) M(t2xy) M(t2yy) \
               M(t3a) M(t3b) M(t3c) M(t3d) M(t4a) M(t4b) M(t4c) M(t4d) M(t4e)
  ALL(GET)
  gal_accumulate(c, o, h);
  ALL(PUT)
#undef ALL
#undef PUT
#undef GET
}

// Galaxy (rho-mixed) and star profile densities of one pair at a pixel
// (value layout): the galaxy pairs in packed two-wide instructions, the
// exponential and de Vaucouleurs sums in the two halves (each half adds its
// components in the order of the derivative kernel's sums).
__device__ __forceinline__ void profiles_value(const float* __restrict__ rec, int ne, int nd,
                                               float px, float py, float& F0, float& F1) {
  const float4* q4 = reinterpret_cast<const float4*>(rec + kCompBase);
  float fs = 0.f;
  float2 f = make_float2(0.f, 0.f);
  const int per = ne + nd;
  const int nb = ne < nd ? ne : nd;
#pragma unroll
  for (int k = 0; k < kPsf; ++k) {
    const Offset o = make_offset(pixel_delta(rec, k, px, py));
    fs += gauss_density(q4[k], o);
    const Offset2 o2 = dup_offset(o);
    const float4* g = q4 + kPsf + k * per;
    for (int j = 0; j < nb; ++j) {
      const float4 a = g[2 * j], b = g[2 * j + 1];
      const float2 arg = fma2(make_float2(a.x, a.y), o2.xx,
                              fma2(make_float2(a.z, a.w), o2.xy,
                                   fma2(make_float2(b.x, b.y), o2.yy, make_float2(b.z, b.w))));
      f = add2(f, make_float2(exp2f(arg.x), exp2f(arg.y)));
    }
    const float4* single = g + 2 * nb;
    for (int j = nb; j < ne; ++j) f.x += gauss_density(*single++, o);
    for (int j = nb; j < nd; ++j) f.y += gauss_density(*single++, o);
  }
  F0 = fmaf(rec[H_RHO], f.x, rec[H_RHO1] * f.y);
  F1 = fs;
}

// profiles_value at two pixels (a and b), each with exactly the
// instructions of profiles_value, reading each staged component once.
__device__ __forceinline__ void profiles_value2(const float* __restrict__ rec, int ne, int nd,
                                                float pxa, float pya, float pxb, float pyb,
                                                float& F0a, float& F1a, float& F0b,
                                                float& F1b) {
  const float4* q4 = reinterpret_cast<const float4*>(rec + kCompBase);
  float fsa = 0.f, fsb = 0.f;
  float2 fa = make_float2(0.f, 0.f), fb = make_float2(0.f, 0.f);
  const int per = ne + nd;
  const int nb = ne < nd ? ne : nd;
#pragma unroll
  for (int k = 0; k < kPsf; ++k) {
    const Offset oa = make_offset(pixel_delta(rec, k, pxa, pya));
    const Offset ob = make_offset(pixel_delta(rec, k, pxb, pyb));
    const float4 qs = q4[k];
    fsa += gauss_density(qs, oa);
    fsb += gauss_density(qs, ob);
    const Offset2 a2 = dup_offset(oa), b2 = dup_offset(ob);
    const float4* g = q4 + kPsf + k * per;
    for (int j = 0; j < nb; ++j) {
      const float4 a = g[2 * j], b = g[2 * j + 1];
      const float2 A11 = make_float2(a.x, a.y), A12 = make_float2(a.z, a.w);
      const float2 A22 = make_float2(b.x, b.y), lw = make_float2(b.z, b.w);
      const float2 ga = fma2(A11, a2.xx, fma2(A12, a2.xy, fma2(A22, a2.yy, lw)));
      const float2 gb = fma2(A11, b2.xx, fma2(A12, b2.xy, fma2(A22, b2.yy, lw)));
      fa = add2(fa, make_float2(exp2f(ga.x), exp2f(ga.y)));
      fb = add2(fb, make_float2(exp2f(gb.x), exp2f(gb.y)));
    }
    const float4* single = g + 2 * nb;
    for (int j = nb; j < ne; ++j, ++single) {
      fa.x += gauss_density(*single, oa);
      fb.x += gauss_density(*single, ob);
    }
    for (int j = nb; j < nd; ++j, ++single) {
      fa.y += gauss_density(*single, oa);
      fb.y += gauss_density(*single, ob);
    }
  }
  const float rho = rec[H_RHO], rho1 = rec[H_RHO1];
  F0a = fmaf(rho, fa.x, rho1 * fa.y);
  F1a = fsa;
  F0b = fmaf(rho, fb.x, rho1 * fb.y);
  F1b = fsb;
}

// The source's own E_q[l f] and V_q[l f] at a pixel.  V uses the
// cancellation-free form sum_i q_i ev_i (k_i F_i)^2 + q0 q1 (k0 F0 - k1 F1)^2.
__device__ __forceinline__ void own_moments(const float* __restrict__ rec, float F0, float F1,
                                            float& Es, float& Vs) {
  const float k0F = rec[H_K0] * F0, k1F = rec[H_K1] * F1;
  Es = fmaf(rec[H_CE0], F0, rec[H_CE1] * F1);
  const float d = k0F - k1F;
  Vs = fmaf(rec[H_Q0] * rec[H_EV0] * k0F, k0F,
            fmaf(rec[H_Q1] * rec[H_EV1] * k1F, k1F, rec[H_Q0] * rec[H_Q1] * d * d));
}

// The 52 Hessian sums of a lane live in its warp's shared memory: row a
// (the sum hidx = kGradAcc + a) of a padded [kHessAcc][33] array, this lane's
// column.  The 33-float rows keep both the per-pixel updates (one row, all
// lanes) and the transposed reduction (one row per lane) free of bank
// conflicts, and the registers this frees keep more warps resident.
constexpr int kHessAcc = kAcc - kGradAcc;   // 52
constexpr int kHessRow = 33;
constexpr int kAccTileF = kAcc * kHessRow;  // all 64 sums at the reduction

struct HessAcc {
  float* __restrict__ col;   // this lane's column of the warp's array
  __device__ __forceinline__ float* at(int idx) const { return col + (idx - kGradAcc) * kHessRow; }
  // sum += v
  __device__ __forceinline__ void add(int idx, float v) const { *at(idx) += v; }
  // sum = fma(a, b, sum)
  __device__ __forceinline__ void fma(int idx, float a, float b) const {
    float* p = at(idx);
    *p = fmaf(a, b, *p);
  }
  // sum = fma(a, b, fma(c, d, sum))
  __device__ __forceinline__ void fma2(int idx, float a, float b, float c, float d) const {
    float* p = at(idx);
    *p = fmaf(a, b, fmaf(c, d, *p));
  }
};

// One pixel: render with derivatives and accumulate value, gradient, Hessian.
__device__ __forceinline__ void pixel_derivs(const float* __restrict__ rec, int ne, int nd,
                                             float px, float py, float x, float2 bg,
                                             float* __restrict__ acc, const HessAcc& hs) {
  // ---- star: value, d mu, d mu d mu
  float F1 = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f, syy = 0.f;
#pragma unroll
  for (int k = 0; k < kPsf; ++k) {
    const Offset o = make_offset(pixel_delta(rec, k, px, py));
    const float* c = rec + kCompBase + k * kStarF;
    const float4 q = *reinterpret_cast<const float4*>(c);
    const float4 pp = *reinterpret_cast<const float4*>(c + 4);
    const float y1 = fmaf(pp.x, o.dx, pp.y * o.dy);
    const float y2 = fmaf(pp.y, o.dx, pp.z * o.dy);
    const float phi = gauss_density(q, o);
    F1 += phi;
    sx = fmaf(phi, y1, sx);
    sy = fmaf(phi, y2, sy);
    sxx = fmaf(phi, fmaf(y1, y1, -pp.x), sxx);
    sxy = fmaf(phi, fmaf(y1, y2, -pp.y), sxy);
    syy = fmaf(phi, fmaf(y2, y2, -pp.z), syy);
  }
  // ---- galaxy: exponential and de Vaucouleurs sums, evaluated in pairs
  GalSums2 g2 = {};
  const int per = ne + nd;
  const int nb = ne < nd ? ne : nd;
  // kept rolled: three copies of this loop cost more in instruction fetch
  // than recomputing the offsets
#pragma unroll 1
  for (int k = 0; k < kPsf; ++k) {
    const float* base = rec + kCompBase + kPsf * kStarF + k * per * kGalF;
    const Offset o = make_offset(pixel_delta(rec, k, px, py));
    const Offset2 o2 = dup_offset(o);
    if (nb == kMaxProf) {
      // the usual eight pairs, unrolled: independent pairs interleave (the
      // loop over PSF components stays rolled: unrolling both measured
      // slower, from instruction fetch)
#pragma unroll
      for (int j = 0; j < kMaxProf; ++j) gal_accumulate2(base + j * 2 * kGalF, o2, g2);
    } else {
      for (int j = 0; j < nb; ++j) gal_accumulate2(base + j * 2 * kGalF, o2, g2);
    }
    const float* single = base + nb * 2 * kGalF;
    for (int j = nb; j < ne; ++j, single += kGalF) gal_single<0>(single, o, g2);
    for (int j = nb; j < nd; ++j, single += kGalF) gal_single<1>(single, o, g2);
  }
  GalSums ge, gd;
#define SPLIT(f) ge.f = g2.f.x; gd.f = g2.f.y;
#define FLIP(f) ge.f = -g2.f.x; gd.f = -g2.f.y;        // odd orders: summed with -y
  SPLIT(s0) FLIP(s1x) FLIP(s1y) SPLIT(s2xx) SPLIT(s2xy) SPLIT(s2yy) SPLIT(t2xx) SPLIT(t2xy)
  SPLIT(t2yy) FLIP(t3a) FLIP(t3b) FLIP(t3c) FLIP(t3d) SPLIT(t4a) SPLIT(t4b) SPLIT(t4c)
  SPLIT(t4d) SPLIT(t4e)
#undef FLIP
#undef SPLIT
  const float rho = rec[H_RHO], rho1 = rec[H_RHO1];
#define MIX(f) fmaf(rho, ge.f, rho1 * gd.f)
  // galaxy density and its derivatives over (mu_x, mu_y, g11, g12, g22, rho)
  const float F0 = MIX(s0);
  float d0[6], h0[6][6];
  d0[0] = MIX(s1x);
  d0[1] = MIX(s1y);
  d0[2] = 0.5f * MIX(t2xx);
  d0[3] = MIX(t2xy);
  d0[4] = 0.5f * MIX(t2yy);
  d0[5] = ge.s0 - gd.s0;
  h0[0][0] = MIX(s2xx);
  h0[0][1] = MIX(s2xy);
  h0[1][1] = MIX(s2yy);
  h0[0][2] = 0.5f * MIX(t3a);
  h0[1][2] = 0.5f * MIX(t3b);
  h0[0][3] = MIX(t3b);
  h0[1][3] = MIX(t3c);
  h0[0][4] = 0.5f * MIX(t3c);
  h0[1][4] = 0.5f * MIX(t3d);
  h0[2][2] = 0.25f * MIX(t4a);
  h0[2][3] = 0.5f * MIX(t4b);
  h0[2][4] = 0.25f * MIX(t4c);
  h0[3][3] = MIX(t4c);
  h0[3][4] = 0.5f * MIX(t4d);
  h0[4][4] = 0.25f * MIX(t4e);
  h0[0][5] = ge.s1x - gd.s1x;
  h0[1][5] = ge.s1y - gd.s1y;
  h0[2][5] = 0.5f * (ge.t2xx - gd.t2xx);
  h0[3][5] = ge.t2xy - gd.t2xy;
  h0[4][5] = 0.5f * (ge.t2yy - gd.t2yy);
  h0[5][5] = 0.f;
#undef MIX

  // ---- moments and the pixel term
  const float cE0 = rec[H_CE0], cE1 = rec[H_CE1], cM0 = rec[H_CM0], cM1 = rec[H_CM1];
  float Es, Vs;
  own_moments(rec, F0, F1, Es, Vs);
  const float bgE = bg.x, bgV = bg.y;
  const float E = bgE + Es, V = bgV + Vs;
  const float r = __frcp_rn(E);
  const float rb = __frcp_rn(bgE);
  const float xr = x * r;
  const float xr2 = xr * r;        // x / E^2
  const float xr3 = xr2 * r;       // x / E^3
  const float TE = fmaf(x - E, r, xr3 * V);
  const float TV = -0.5f * xr2;
  const float TEE = fmaf(-3.f * xr3 * r, V, -xr2);
  const float TEV = xr3;
  const float tE = fmaf(-2.f * Es, TV, TE);
  const float tM = TV;
  const float tEE = fmaf(-4.f * Es, TEV, fmaf(-2.f, TV, TEE));
  const float tEM = TEV;

  acc[0] += fmaf(x, log1pf(Es * rb) - 0.5f * V * r * r + 0.5f * bgV * rb * rb, -Es);
  acc[1] += fmaf(x, __logf(bgE) - 0.5f * bgV * rb * rb, -bgE);

  // gradient vectors of E_s (a) and M_s (b) over the six geometric coordinates
  float aG[6], bG[6];
  const float m0 = 2.f * cM0 * F0, m1 = 2.f * cM1 * F1;
  aG[0] = fmaf(cE0, d0[0], cE1 * sx);
  aG[1] = fmaf(cE0, d0[1], cE1 * sy);
  bG[0] = fmaf(m0, d0[0], m1 * sx);
  bG[1] = fmaf(m0, d0[1], m1 * sy);
#pragma unroll
  for (int g = 2; g < 6; ++g) {
    aG[g] = cE0 * d0[g];
    bG[g] = m0 * d0[g];
  }
  const float F0s = F0 * F0, F1s = F1 * F1;
  // gradient over w
  acc[2] = fmaf(tE, F0, acc[2]);
  acc[3] = fmaf(tE, F1, acc[3]);
  acc[4] = fmaf(tM, F0s, acc[4]);
  acc[5] = fmaf(tM, F1s, acc[5]);
#pragma unroll
  for (int g = 0; g < 6; ++g) acc[6 + g] = fmaf(tE, aG[g], fmaf(tM, bG[g], acc[6 + g]));

  // Hessian: tEE a a^T + tEM (a b^T + b a^T) + tE d2E_s + tM d2M_s
  float u[6], cg[6];
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    cg[g] = tEM * bG[g];
    u[g] = fmaf(tEE, aG[g], cg[g]);
  }
  hs.fma(hidx(0, 0), tEE, F0s);
  hs.fma(hidx(0, 1), tEE, F0 * F1);
  hs.fma(hidx(1, 1), tEE, F1s);
  hs.fma(hidx(0, 2), tEM * F0, F0s);
  hs.fma(hidx(0, 3), tEM * F0, F1s);
  hs.fma(hidx(1, 2), tEM * F1, F0s);
  hs.fma(hidx(1, 3), tEM * F1, F1s);
  const float tm2F0 = 2.f * tM * F0, tm2F1 = 2.f * tM * F1;
  const float eF0 = tEM * F0s, eF1 = tEM * F1s;
#pragma unroll
  for (int g = 0; g < 6; ++g) {
    hs.fma2(hidx(0, 4 + g), F0, u[g], tE, d0[g]);
    hs.fma2(hidx(2, 4 + g), eF0, aG[g], tm2F0, d0[g]);
  }
  hs.fma2(hidx(1, 4), F1, u[0], tE, sx);
  hs.fma2(hidx(1, 5), F1, u[1], tE, sy);
  hs.fma2(hidx(3, 4), eF1, aG[0], tm2F1, sx);
  hs.fma2(hidx(3, 5), eF1, aG[1], tm2F1, sy);
#pragma unroll
  for (int g = 2; g < 6; ++g) {
    hs.fma(hidx(1, 4 + g), F1, u[g]);
    hs.fma(hidx(3, 4 + g), eF1, aG[g]);
  }
  const float D0 = fmaf(tE, cE0, tM * m0);   // dl/dF0 (direct part)
  const float D1 = fmaf(tE, cE1, tM * m1);
  const float q0 = 2.f * tM * cM0, q1 = 2.f * tM * cM1;
  const float h1[2][2] = {{sxx, sxy}, {sxy, syy}};
  const float d1[2] = {sx, sy};
#pragma unroll
  for (int g = 0; g < 6; ++g) {
#pragma unroll
    for (int h = g; h < 6; ++h) {
      float v = fmaf(aG[g], u[h], cg[g] * aG[h]);
      v = fmaf(D0, h0[g][h], v);
      v = fmaf(q0 * d0[g], d0[h], v);
      if (g < 2 && h < 2) {
        v = fmaf(D1, h1[g][h], v);
        v = fmaf(q1 * d1[g], d1[h], v);
      }
      hs.add(hidx(4 + g, 4 + h), v);
    }
  }
}

// Gradient-only sums of one galaxy profile: value, d mu, and the
// tau-weighted second order for dG (the heat equation again).
struct GalSums1 {
  float s0, s1x, s1y, t2xx, t2xy, t2yy;
};

__device__ __forceinline__ void gal_accumulate1(const float* __restrict__ c, const Offset& o,
                                                GalSums1& g) {
  const float4 q = *reinterpret_cast<const float4*>(c);
  const float4 pp = *reinterpret_cast<const float4*>(c + 4);
  const float nP11 = pp.x, nP12 = pp.y, nP22 = pp.z;
  const float z1 = fmaf(nP11, o.dx, nP12 * o.dy);       // -y1
  const float z2 = fmaf(nP12, o.dx, nP22 * o.dy);
  const float phi = gauss_density(q, o);
  const float pt = phi * pp.w;
  g.s0 += phi;
  g.s1x = fmaf(phi, z1, g.s1x);
  g.s1y = fmaf(phi, z2, g.s1y);
  g.t2xx = fmaf(pt, fmaf(z1, z1, nP11), g.t2xx);
  g.t2xy = fmaf(pt, fmaf(z1, z2, nP12), g.t2xy);
  g.t2yy = fmaf(pt, fmaf(z2, z2, nP22), g.t2yy);
}

struct GalSums1x2 {
  float2 s0, s1x, s1y, t2xx, t2xy, t2yy;
};

// gal_accumulate1 on a staged pair (exponential in the even slots).
__device__ __forceinline__ void gal_accumulate1x2(const float* __restrict__ c, const Offset2& o,
                                                  GalSums1x2& g) {
  const float4 qa = *reinterpret_cast<const float4*>(c);
  const float4 qb = *reinterpret_cast<const float4*>(c + 4);
  const float4 pa = *reinterpret_cast<const float4*>(c + 8);
  const float4 pb = *reinterpret_cast<const float4*>(c + 12);
  const float2 A11 = make_float2(qa.x, qa.y), A12 = make_float2(qa.z, qa.w);
  const float2 A22 = make_float2(qb.x, qb.y), lw = make_float2(qb.z, qb.w);
  const float2 nP11 = make_float2(pa.x, pa.y), nP12 = make_float2(pa.z, pa.w);
  const float2 nP22 = make_float2(pb.x, pb.y), tau = make_float2(pb.z, pb.w);
  const float2 z1 = fma2(nP11, o.dx, mul2(nP12, o.dy));
  const float2 z2 = fma2(nP12, o.dx, mul2(nP22, o.dy));
  const float2 arg = fma2(A11, o.xx, fma2(A12, o.xy, fma2(A22, o.yy, lw)));
  const float2 phi = make_float2(exp2f(arg.x), exp2f(arg.y));
  const float2 pt = mul2(phi, tau);
  g.s0 = add2(g.s0, phi);
  g.s1x = fma2(phi, z1, g.s1x);
  g.s1y = fma2(phi, z2, g.s1y);
  g.t2xx = fma2(pt, fma2(z1, z1, nP11), g.t2xx);
  g.t2xy = fma2(pt, fma2(z1, z2, nP12), g.t2xy);
  g.t2yy = fma2(pt, fma2(z2, z2, nP22), g.t2yy);
}

template <int L>
__device__ __forceinline__ void gal_single1(const float* __restrict__ c, const Offset& o,
                                            GalSums1x2& g) {
  GalSums1 h;
#define GET(f) h.f = L ? g.f.y : g.f.x;
#define PUT(f) (L ? g.f.y : g.f.x) = h.f;
#define ALL(M) M(s0) M(s1x) M(s1y) M(t2xx) M(t2xy) M(t2yy)
  ALL(GET)
  gal_accumulate1(c, o, h);
  ALL(PUT)
#undef ALL
#undef PUT
#undef GET
}

// One pixel, value and gradient only (the adjoint of the pixel term through
// E_s and M_s onto the per-image natural coordinates): 12 accumulators.
__device__ __forceinline__ void pixel_grad(const float* __restrict__ rec, int ne, int nd,
                                           float px, float py, float x, float2 bg,
                                           float* __restrict__ acc) {
  float F1 = 0.f, sx = 0.f, sy = 0.f;
  float2 dk[kPsf];
#pragma unroll
  for (int k = 0; k < kPsf; ++k) {
    dk[k] = pixel_delta(rec, k, px, py);
    const Offset o = make_offset(dk[k]);
    const float* c = rec + kCompBase + k * kStarF;
    const float4 q = *reinterpret_cast<const float4*>(c);
    const float4 pp = *reinterpret_cast<const float4*>(c + 4);
    const float y1 = fmaf(pp.x, o.dx, pp.y * o.dy);
    const float y2 = fmaf(pp.y, o.dx, pp.z * o.dy);
    const float phi = gauss_density(q, o);
    F1 += phi;
    sx = fmaf(phi, y1, sx);
    sy = fmaf(phi, y2, sy);
  }
  GalSums1x2 g2 = {};
  const int per = ne + nd;
  const int nb = ne < nd ? ne : nd;
#pragma unroll
  for (int k = 0; k < kPsf; ++k) {
    const float* base = rec + kCompBase + kPsf * kStarF + k * per * kGalF;
    const Offset o = make_offset(dk[k]);
    const Offset2 o2 = dup_offset(o);
    for (int j = 0; j < nb; ++j) gal_accumulate1x2(base + j * 2 * kGalF, o2, g2);
    const float* single = base + nb * 2 * kGalF;
    for (int j = nb; j < ne; ++j, single += kGalF) gal_single1<0>(single, o, g2);
    for (int j = nb; j < nd; ++j, single += kGalF) gal_single1<1>(single, o, g2);
  }
  GalSums1 ge, gd;
#define SPLIT(f) ge.f = g2.f.x; gd.f = g2.f.y;
#define FLIP(f) ge.f = -g2.f.x; gd.f = -g2.f.y;        // first order: summed with -y
  SPLIT(s0) FLIP(s1x) FLIP(s1y) SPLIT(t2xx) SPLIT(t2xy) SPLIT(t2yy)
#undef FLIP
#undef SPLIT
  const float rho = rec[H_RHO], rho1 = rec[H_RHO1];
#define MIX(f) fmaf(rho, ge.f, rho1 * gd.f)
  const float F0 = MIX(s0);
  float d0[6];
  d0[0] = MIX(s1x);
  d0[1] = MIX(s1y);
  d0[2] = 0.5f * MIX(t2xx);
  d0[3] = MIX(t2xy);
  d0[4] = 0.5f * MIX(t2yy);
  d0[5] = ge.s0 - gd.s0;
#undef MIX
  const float cE0 = rec[H_CE0], cE1 = rec[H_CE1], cM0 = rec[H_CM0], cM1 = rec[H_CM1];
  float Es, Vs;
  own_moments(rec, F0, F1, Es, Vs);
  const float bgE = bg.x, bgV = bg.y;
  const float E = bgE + Es, V = bgV + Vs;
  const float r = __frcp_rn(E);
  const float rb = __frcp_rn(bgE);
  const float xr2 = x * r * r;
  const float TE = fmaf(x - E, r, xr2 * r * V);
  const float TV = -0.5f * xr2;
  const float tE = fmaf(-2.f * Es, TV, TE);
  const float tM = TV;
  acc[0] += fmaf(x, log1pf(Es * rb) - 0.5f * V * r * r + 0.5f * bgV * rb * rb, -Es);
  acc[1] += fmaf(x, __logf(bgE) - 0.5f * bgV * rb * rb, -bgE);
  const float m0 = 2.f * cM0 * F0, m1 = 2.f * cM1 * F1;
  acc[2] = fmaf(tE, F0, acc[2]);
  acc[3] = fmaf(tE, F1, acc[3]);
  acc[4] = fmaf(tM, F0 * F0, acc[4]);
  acc[5] = fmaf(tM, F1 * F1, acc[5]);
  const float a0 = fmaf(cE0, d0[0], cE1 * sx), a1 = fmaf(cE0, d0[1], cE1 * sy);
  const float b0 = fmaf(m0, d0[0], m1 * sx), b1 = fmaf(m0, d0[1], m1 * sy);
  acc[6] = fmaf(tE, a0, fmaf(tM, b0, acc[6]));
  acc[7] = fmaf(tE, a1, fmaf(tM, b1, acc[7]));
  const float cg = fmaf(tE, cE0, tM * m0);
#pragma unroll
  for (int g = 2; g < 6; ++g) acc[6 + g] = fmaf(cg, d0[g], acc[6 + g]);
}

// Warp-shared memory of the derivative kernel: the staged record, then the
// [kAcc][kHessRow] sums (rows 0..51 the Hessian sums, rows 52..63 the value
// and gradient sums, written there for the final reduction).
constexpr int kDerivWarpF = kDerivRecF + kAccTileF;


// Adds the 64 sums of an item over the warp's lanes and writes them.  The
// two value sums take the shuffle tree every pixel kernel uses for its value
// sums, so that the value of an evaluation is the same in every pass (the
// trust-region ratio compares values of the derivative and value passes);
// for the other 62, lane l adds up rows (sums l and l + 32) along the
// 33-float rows, in lane order, four chains per row.
__device__ __forceinline__ void reduce_tile(float* __restrict__ tile, float* __restrict__ acc,
                                            float* __restrict__ out, int lane) {
#pragma unroll
  for (int a = 2; a < kGradAcc; ++a) tile[(kHessAcc + a) * kHessRow + lane] = acc[a];
  const float v0 = warp_sum(acc[0]), v1 = warp_sum(acc[1]);
  if (lane == 0) {
    out[0] = v0;
    out[1] = v1;
  }
  __syncwarp();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int o = lane + 32 * h;
    if (o < 2) continue;
    const int row = o < kGradAcc ? kHessAcc + o : o - kGradAcc;
    const float* r = tile + row * kHessRow;
    float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll
    for (int k = 0; k < 32; k += 4) {
      c0 += r[k];
      c1 += r[k + 1];
      c2 += r[k + 2];
      c3 += r[k + 3];
    }
    out[o] = (c0 + c1) + (c2 + c3);
  }
}

// Four blocks of four warps per SM: with the Hessian sums in shared memory
// the kernel fits 128 registers a thread, and 16 warps keep the FP32 pipe
// fed.  (Forming the background here instead of in background_kernel was
// measured slower: the cached-moment loads inside the pixel loop stall 16
// warps more than a separate kernel's many warps.)
template <bool kQueue>
__global__ void __launch_bounds__(128, 4) derivs_kernel(PlanView v, int ne, int nd) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kDerivWarpF;
  float* tile = rec + kDerivRecF;
  const HessAcc hs{tile + lane};
  WarpQueue wq(kQueue ? v.work_ctr : nullptr);
  for (; wq.it < v.n_items; wq.advance()) {
    wq.ask(lane);
    const int it = wq.it;
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    if (!v.active[pi.slot]) continue;
    __syncwarp();
    stage_record<true>(rec, v.records + (size_t)item.pair * kRecF,
                       kPsf * (1 + ne + nd), lane, ne);
#pragma unroll
    for (int a = 0; a < kHessAcc; ++a) tile[a * kHessRow + lane] = 0.f;
    __syncwarp();
    float acc[kGradAcc];
#pragma unroll
    for (int a = 0; a < kGradAcc; ++a) acc[a] = 0.f;
    const int end = item.start + item.count;
    PixelWalk pw(item.start + lane, pi.w);
    for (int q = item.start + lane; q < end; q += 32, pw.next(pi.w)) {
      const int qy = pw.qy, qx = pw.qx;
      const float x = __ldg(v.pixels + pi.pix_base + (int64_t)qy * pi.stride + qx);
      const float2 bg = v.bg[pi.bg_base + q];
      pixel_derivs(rec, ne, nd, (float)qx, (float)qy, x, bg, acc, hs);
    }
    __syncwarp();
    reduce_tile(tile, acc, v.partials + (size_t)it * kAcc, lane);
  }
  wq.done(lane);
}

template <bool kQueue>
__global__ void __launch_bounds__(128) grad_kernel(PlanView v, int ne, int nd) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kDerivRecF;
  WarpQueue wq(kQueue ? v.work_ctr : nullptr);
  for (; wq.it < v.n_items; wq.advance()) {
    wq.ask(lane);
    const int it = wq.it;
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    if (!v.active[pi.slot]) continue;
    __syncwarp();
    stage_record<true>(rec, v.records + (size_t)item.pair * kRecF,
                       kPsf * (1 + ne + nd), lane, ne);
    __syncwarp();
    float acc[kGradAcc];
#pragma unroll
    for (int a = 0; a < kGradAcc; ++a) acc[a] = 0.f;
    const int end = item.start + item.count;
    PixelWalk pw(item.start + lane, pi.w);
    for (int q = item.start + lane; q < end; q += 32, pw.next(pi.w)) {
      const int qy = pw.qy, qx = pw.qx;
      const float x = __ldg(v.pixels + pi.pix_base + (int64_t)qy * pi.stride + qx);
      const float2 bg = v.bg[pi.bg_base + q];
      pixel_grad(rec, ne, nd, (float)qx, (float)qy, x, bg, acc);
    }
#pragma unroll
    for (int a = 0; a < kGradAcc; ++a) acc[a] = warp_sum(acc[a]);
    float* out = v.partials + (size_t)it * kAcc;
#pragma unroll
    for (int a = 0; a < kGradAcc; ++a)
      if (a == lane) out[a] = acc[a];
  }
  wq.done(lane);
}

// Value-only pass over one item: the pixel term at the record's point
// (relative and baseline sums into the item's slot of vpartials); with
// render set, the own moments are also stored there (row-major over the
// patch, item pixels only).
__device__ __forceinline__ void value_item(const PlanView& v, int it, const Item& item,
                                           const PairInfo& pi, float* rec, int lane, int ne,
                                           int nd, float2* render) {
  __syncwarp();
  stage_record<false>(rec, v.records + (size_t)item.pair * kRecF, kPsf * (1 + ne + nd), lane, ne);
  __syncwarp();
  float rel = 0.f, base = 0.f;
  const int end = item.start + item.count;
  // a lane's pixels q and q + 32 in one pass over the staged components; the
  // sums take pixel q, then q + 32, as one pixel per pass would
  PixelWalk pa(item.start + lane, pi.w, 64), pb(item.start + lane + 32, pi.w, 64);
  for (int q = item.start + lane; q < end; q += 64, pa.next(pi.w), pb.next(pi.w)) {
    const bool has_b = q + 32 < end;
    float F0[2], F1[2];
    profiles_value2(rec, ne, nd, (float)pa.qx, (float)pa.qy, (float)pb.qx, (float)pb.qy, F0[0],
                    F1[0], F0[1], F1[1]);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && !has_b) break;
      const int qq = q + 32 * h, qx = h ? pb.qx : pa.qx, qy = h ? pb.qy : pa.qy;
      const float x = __ldg(v.pixels + pi.pix_base + (int64_t)qy * pi.stride + qx);
      const float2 bg = v.bg[pi.bg_base + qq];
      float Es, Vs;
      own_moments(rec, F0[h], F1[h], Es, Vs);
      if (render) render[qq] = make_float2(Es, Vs);
      const float E = bg.x + Es, V = bg.y + Vs;
      const float r = __frcp_rn(E), rb = __frcp_rn(bg.x);
      rel += fmaf(x, log1pf(Es * rb) - 0.5f * V * r * r + 0.5f * bg.y * rb * rb, -Es);
      base += fmaf(x, __logf(bg.x) - 0.5f * bg.y * rb * rb, -bg.x);
    }
  }
  rel = warp_sum(rel);
  base = warp_sum(base);
  if (lane == 0) {
    v.vpartials[2 * (size_t)it] = rel;
    v.vpartials[2 * (size_t)it + 1] = base;
  }
}

// keep_render: 0 none; 1 the own moments into v.trial_render; 2 into the
// source's other half of the render cache (where a Newton step's trial
// render waits for the accept rule).
// Eight blocks per SM (64 registers): 3.5 % faster than seven at 72.
template <bool kQueue>
__global__ void __launch_bounds__(128, 8) value_kernel(PlanView v, int ne, int nd,
                                                    int keep_render) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  WarpQueue wq(kQueue ? v.work_ctr : nullptr);
  for (; wq.it < v.n_items; wq.advance()) {
    wq.ask(lane);
    const int it = wq.it;
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    if (!v.active[pi.slot]) continue;
    float2* render = nullptr;
    if (keep_render == 1) {
      render = v.trial_render + pi.bg_base;
    } else if (keep_render == 2) {
      const int64_t other = cache_base(v, pi.source) ? 0 : v.cache_n_pool;
      render = v.cache + other + v.patches[pi.patch].pool_offset;
    }
    value_item(v, it, item, pi, rec, lane, ne, nd, render);
  }
  wq.done(lane);
}

// Stages neighbour pairs [c0, c0 + cnt) of own pair pi: rectangle and offset
// of the neighbour's patch in the render cache (in its current half).
__device__ __forceinline__ void stage_neighbours(const PlanView& v, const PairInfo& pi, int c0,
                                                 int cnt, int4* srect, int64_t* soff, int lane) {
  if (lane < cnt) {
    const PairInfo qn = v.pairs[v.pair_nbr[pi.nbr_begin + c0 + lane]];
    srect[lane] = make_int4(qn.x0, qn.y0, qn.w, qn.h);
    soff[lane] = v.patches[qn.patch].pool_offset + cache_base(v, qn.source);
  }
}

// Adds the cached moments of the staged neighbours whose patches hold the
// pixel (gx, gy) of the image, in staging order.
__device__ __forceinline__ float2 add_neighbours(const PlanView& v, float2 b, int gx, int gy,
                                                 int cnt, const int4* srect,
                                                 const int64_t* soff) {
  for (int k = 0; k < cnt; ++k) {
    const int4 r = srect[k];
    const int lx = gx - r.x, ly = gy - r.y;
    if (lx < 0 || ly < 0 || lx >= r.z || ly >= r.w) continue;
    const float2 c = v.cache[soff[k] + ly * r.z + lx];
    b.x += c.x;
    b.y += c.y;
  }
  return b;
}

// Background of item it's pixels (own pair pi): sky plus each neighbour's E
// and V where the pixel lies in that neighbour's patch (support rule, Sec.
// 2.2.3).  rec: the warp's staging area (kValRecF floats).
__device__ __forceinline__ void background_item(const PlanView& v, const Item& item,
                                                const PairInfo& pi, float* rec, int lane, int ne,
                                                int nd) {
  const celeste_image& im = v.images[pi.image];
  const int end = item.start + item.count;
  if (v.cache) {
    // sky plus the neighbours' cached moments (the values the render
    // below would produce, added in the same order), 32 neighbour pairs
    // at a time staged in the warp's shared memory; the first 32 are
    // added in the pass that evaluates the sky
    int4* srect = reinterpret_cast<int4*>(rec);
    int64_t* soff = reinterpret_cast<int64_t*>(rec + 4 * 32);
    const int nn = pi.nbr_end - pi.nbr_begin;
    for (int c0 = 0; c0 == 0 || c0 < nn; c0 += 32) {
      const int cnt = max(0, min(32, nn - c0));
      __syncwarp();
      stage_neighbours(v, pi, c0, cnt, srect, soff, lane);
      __syncwarp();
      PixelWalk pw(item.start + lane, pi.w);
      for (int q = item.start + lane; q < end; q += 32, pw.next(pi.w)) {
        const int gx = pi.x0 + pw.qx, gy = pi.y0 + pw.qy;
        float2 b;
        if (c0 == 0) {
          const float s = sky_value(im, v.sky, (float)gx, (float)gy);
          if (!(s > 0.f)) set_error(v.err, CELESTE_DERR_SKY);
          b = make_float2(s, 0.f);
        } else {
          b = v.bg[pi.bg_base + q];
        }
        v.bg[pi.bg_base + q] = add_neighbours(v, b, gx, gy, cnt, srect, soff);
      }
    }
    return;
  }
  PixelWalk pw(item.start + lane, pi.w);
  for (int q = item.start + lane; q < end; q += 32, pw.next(pi.w)) {
    const float s = sky_value(im, v.sky, (float)(pi.x0 + pw.qx), (float)(pi.y0 + pw.qy));
    if (!(s > 0.f)) set_error(v.err, CELESTE_DERR_SKY);
    v.bg[pi.bg_base + q] = make_float2(s, 0.f);
  }
  for (int nb = pi.nbr_begin; nb < pi.nbr_end; ++nb) {
    const int np = v.pair_nbr[nb];
    const PairInfo qn = v.pairs[np];
    __syncwarp();
    stage_record<false>(rec, v.records + (size_t)np * kRecF, kPsf * (1 + ne + nd), lane, ne);
    __syncwarp();
    for (int q = item.start + lane; q < end; q += 32) {
      const int qy = q / pi.w;
      const int gx = pi.x0 + (q - qy * pi.w), gy = pi.y0 + qy;
      const int lx = gx - qn.x0, ly = gy - qn.y0;
      if (lx < 0 || ly < 0 || lx >= qn.w || ly >= qn.h) continue;
      float F0, F1, Es, Vs;
      profiles_value(rec, ne, nd, (float)lx, (float)ly, F0, F1);
      own_moments(rec, F0, F1, Es, Vs);
      float2 b = v.bg[pi.bg_base + q];
      b.x += Es;
      b.y += Vs;
      v.bg[pi.bg_base + q] = b;
    }
  }
}

__global__ void __launch_bounds__(128) background_kernel(PlanView v, int ne, int nd) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  WarpQueue wq(nullptr);   // grid stride (short units, as in prepare_kernel)
  for (; wq.it < v.n_items; wq.advance()) {
    wq.ask(lane);
    const Item item = v.items[wq.it];
    const PairInfo pi = v.pairs[item.pair];
    if (!v.active[pi.slot]) continue;
    background_item(v, item, pi, rec, lane, ne, nd);
  }
  wq.done(lane);
}

// The start of a Newton iteration of a colour class, one warp per unit of
// work: the active set from the sources' status (a warp per 32 slots), the
// records of pairs [0, n_setup) at theta, and, with bg set, the background
// of every item of an active slot (the render cache supplies the
// neighbours, so the own records are all it needs).
__global__ void __launch_bounds__(128) prepare_kernel(PlanView v, const ModelDev* __restrict__ model,
                                                      const int32_t* __restrict__ status,
                                                      int n_setup, int bg, int ne, int nd) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  const int n_mark = (v.n + 31) / 32;
  const int units = n_mark + n_setup + (bg ? v.n_items : 0);
  // grid stride: its units are short, so a queue's claim would not return
  // before the next unit (measured 11 % slower)
  WarpQueue wq(nullptr);
  for (; wq.it < units; wq.advance()) {
    wq.ask(lane);
    const int u = wq.it;
    if (u < n_mark) {
      const int j = 32 * u + lane;
      if (j < v.n) v.active[j] = active_of(status[v.src_ids[j]]);
    } else if (u < n_mark + n_setup) {
      setup_pair(v, model, u - n_mark, false, rec, rec + 32, lane);
    } else {
      const Item item = v.items[u - n_mark - n_setup];
      const PairInfo pi = v.pairs[item.pair];
      if (!active_of(status[pi.source])) continue;
      background_item(v, item, pi, rec, lane, ne, nd);
    }
  }
  wq.done(lane);
}

// Own E_s and V_s of every plan pair, scattered to the caller's pool layout.
__global__ void __launch_bounds__(128) render_kernel(PlanView v, int ne, int nd, float* E_out,
                                                     float* V_out,
                                                     const celeste_patch* __restrict__ patches) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = blockIdx.x * (blockDim.x >> 5) + wib; it < v.n_items; it += nwarps) {
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    const int64_t off = patches[pi.patch].pool_offset;
    __syncwarp();
    stage_record<false>(rec, v.records + (size_t)item.pair * kRecF,
                        kPsf * (1 + ne + nd), lane, ne);
    __syncwarp();
    const int end = item.start + item.count;
    for (int q = item.start + lane; q < end; q += 32) {
      const int qy = q / pi.w;
      const int qx = q - qy * pi.w;
      float F0, F1, Es, Vs;
      profiles_value(rec, ne, nd, (float)qx, (float)qy, F0, F1);
      own_moments(rec, F0, F1, Es, Vs);
      if (E_out) E_out[off + q] = Es;
      if (V_out) V_out[off + q] = Vs;
    }
  }
}

// Own E_s and V_s of the plan's pairs into the problem's render cache.
__global__ void __launch_bounds__(128) render_cache_kernel(PlanView v, int ne, int nd,
                                                           const int32_t* __restrict__ status) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = blockIdx.x * (blockDim.x >> 5) + wib; it < v.n_items; it += nwarps) {
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    if (status && status[pi.source] != CELESTE_ST_ACCEPTED) continue;
    float2* out = v.cache + cache_base(v, pi.source) + v.patches[pi.patch].pool_offset;
    __syncwarp();
    stage_record<false>(rec, v.records + (size_t)item.pair * kRecF,
                        kPsf * (1 + ne + nd), lane, ne);
    __syncwarp();
    const int end = item.start + item.count;
    for (int q = item.start + lane; q < end; q += 32) {
      const int qy = q / pi.w;
      const int qx = q - qy * pi.w;
      float F0, F1, Es, Vs;
      profiles_value(rec, ne, nd, (float)qx, (float)qy, F0, F1);
      own_moments(rec, F0, F1, Es, Vs);
      out[q] = make_float2(Es, Vs);
    }
  }
}

// A copy: every lane loads up to eight pixels before it stores any, so that
// enough loads are in flight to approach the copy bandwidth.
__global__ void __launch_bounds__(128) commit_render_kernel(PlanView v,
                                                            const int32_t* __restrict__ status) {
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < v.n_items; it += nwarps) {
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    if (status[pi.source] != CELESTE_ST_ACCEPTED) continue;
    const float2* __restrict__ src = v.trial_render + pi.bg_base + item.start;
    float2* __restrict__ dst =
        v.cache + cache_base(v, pi.source) + v.patches[pi.patch].pool_offset + item.start;
    const int n = item.count;
    for (int q0 = lane; q0 < n; q0 += 8 * 32) {
      float2 r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + 32 * u < n) r[u] = __ldcs(src + q0 + 32 * u);
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (q0 + 32 * u < n) dst[q0 + 32 * u] = r[u];
    }
  }
}

// Adds the plan's own moments into per-image buffers in the pixel-pool
// layout.  Plain read-modify-write: sources of one colour class never share
// a pixel, and classes are launched one after another.
__global__ void __launch_bounds__(128) accumulate_kernel(PlanView v, int ne, int nd, float* Eimg,
                                                         float* Vimg) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  float* rec = smem + wib * kValRecF;
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  for (int it = blockIdx.x * (blockDim.x >> 5) + wib; it < v.n_items; it += nwarps) {
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    __syncwarp();
    stage_record<false>(rec, v.records + (size_t)item.pair * kRecF,
                        kPsf * (1 + ne + nd), lane, ne);
    __syncwarp();
    const int end = item.start + item.count;
    for (int q = item.start + lane; q < end; q += 32) {
      const int qy = q / pi.w;
      const int qx = q - qy * pi.w;
      float F0, F1, Es, Vs;
      profiles_value(rec, ne, nd, (float)qx, (float)qy, F0, F1);
      own_moments(rec, F0, F1, Es, Vs);
      const int64_t m = pi.pix_base + (int64_t)qy * pi.stride + qx;
      Eimg[m] += Es;
      Vimg[m] += Vs;
    }
  }
}

// Pixel term -E + x (log E - V / (2 E^2)) (Eq. eq:log_p_last, without
// log x!) over every pixel of image blockIdx.y, with E = sky + Eimg and
// V = Vimg; compensated FP32 sums per thread, FP64 across threads; one
// partial per block in parts[blockIdx.y * gridDim.x + blockIdx.x].
__global__ void __launch_bounds__(256) field_term_kernel(const celeste_image* __restrict__ images,
                                                         const float* __restrict__ pixels,
                                                         const float* __restrict__ sky,
                                                         const float* __restrict__ Eimg,
                                                         const float* __restrict__ Vimg,
                                                         unsigned int* err, double* parts) {
  const celeste_image& im = images[blockIdx.y];
  const int64_t n = (int64_t)im.height * im.width;
  float s = 0.f, c = 0.f;
  for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n;
       f += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(f / im.width), x = (int)(f - (int64_t)y * im.width);
    const int64_t m = im.pix_offset + (int64_t)y * im.row_stride + x;
    const float sk = sky_value(im, sky, (float)x, (float)y);
    if (!(sk > 0.f)) set_error(err, CELESTE_DERR_SKY);
    const float E = sk + Eimg[m], V = Vimg[m], cnt = pixels[m];
    const float r = __frcp_rn(E);
    const float t = fmaf(cnt, __logf(E) - 0.5f * V * r * r, -E);
    const float yk = t - c;
    const float tk = s + yk;
    c = (tk - s) - yk;
    s = tk;
  }
  double d = (double)s - (double)c;
  d = warp_sum_d(d);
  __shared__ double red[8];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += red[w];
    parts[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
  }
}

// out[0] = sum parts - sum kl; out[1] = sum parts; out[2] = sum kl (fixed
// order, one block).
__global__ void __launch_bounds__(256) field_sum_kernel(const double* parts, int n_parts,
                                                        const double* kl, int n_kl, double* out) {
  __shared__ double red[2][256];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n_parts; i += blockDim.x) a += parts[i];
  for (int i = threadIdx.x; i < n_kl; i += blockDim.x) b += kl[i];
  red[0][threadIdx.x] = a;
  red[1][threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      red[0][threadIdx.x] += red[0][threadIdx.x + w];
      red[1][threadIdx.x] += red[1][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[1] = red[0][0];
    out[2] = red[1][0];
    out[0] = red[0][0] - red[1][0];
  }
}

__global__ void bg_scatter_kernel(PlanView v, float* bgE, float* bgV,
                                  const celeste_patch* __restrict__ patches) {
  const int nwarps = gridDim.x * (blockDim.x >> 5);
  const int lane = threadIdx.x & 31;
  for (int it = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; it < v.n_items; it += nwarps) {
    const Item item = v.items[it];
    const PairInfo pi = v.pairs[item.pair];
    const int64_t off = patches[pi.patch].pool_offset;
    for (int q = item.start + lane; q < item.start + item.count; q += 32) {
      const float2 b = v.bg[pi.bg_base + q];
      if (bgE) bgE[off + q] = b.x;
      if (bgV) bgV[off + q] = b.y;
    }
  }
}

static size_t smem_bytes(int wpb) { return (size_t)wpb * kValRecF * sizeof(float); }
static size_t smem_bytes_derivs(int wpb) { return (size_t)wpb * kDerivWarpF * sizeof(float); }
static size_t smem_bytes_grad(int wpb) { return (size_t)wpb * kDerivRecF * sizeof(float); }

constexpr int kWpb = 4;   // warps per block of the pixel kernels

// The derivative kernel's dynamic shared memory is close to the default 48 KB
// limit: raise the limit to what it uses.
static DeviceOnce g_derivs_attr;
static cudaError_t derivs_attr() {
  return g_derivs_attr.run([] {
    cudaError_t e = cudaFuncSetAttribute(derivs_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes_derivs(kWpb));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(derivs_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem_bytes_derivs(kWpb));
    return e;
  });
}

// Resident blocks per SM of each persistent pixel kernel, per device (0
// until measured on that device).
enum {
  kOccDerivs, kOccGrad, kOccValue, kOccDerivsQ, kOccGradQ, kOccValueQ, kOccBackground, kOccRender,
  kOccCommit, kOccPrepare, kOccKinds
};
static std::atomic<int> g_occ[kMaxDevices][kOccKinds] = {};
static DeviceOnce g_occ_once;

cudaError_t init_pixel_occupancy() {
  if (cudaError_t e = derivs_attr()) return e;
  return g_occ_once.run([] {
    const int dev = current_device();
    const size_t sm = smem_bytes(kWpb);
    int occ[kOccKinds] = {};
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &occ[kOccDerivs], derivs_kernel<false>, kWpb * 32, smem_bytes_derivs(kWpb));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccDerivsQ], derivs_kernel<true>,
                                                        kWpb * 32, smem_bytes_derivs(kWpb));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccGrad], grad_kernel<false>,
                                                        kWpb * 32, smem_bytes_grad(kWpb));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccGradQ], grad_kernel<true>,
                                                        kWpb * 32, smem_bytes_grad(kWpb));
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccValue], value_kernel<false>,
                                                        kWpb * 32, sm);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccValueQ], value_kernel<true>,
                                                        kWpb * 32, sm);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccBackground], background_kernel,
                                                        kWpb * 32, sm);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccRender], render_cache_kernel,
                                                        kWpb * 32, sm);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccCommit], commit_render_kernel,
                                                        kWpb * 32, 0);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ[kOccPrepare], prepare_kernel,
                                                        kWpb * 32, sm);
    if (e == cudaSuccess)
      for (int k = 0; k < kOccKinds; ++k) g_occ[dev][k].store(occ[k], std::memory_order_relaxed);
    return e;
  });
}

// Persistent grid: SMs x (the tuning's blocks per SM, else the kernel's
// occupancy on the current device), no more blocks than the work needs.
static int grid_for(const Launch& L, int n_items, int wpb, int occ_kind = -1) {
  int per_sm = L.blocks_per_sm;
  if (per_sm <= 0) {
    const int occ =
        occ_kind >= 0 ? g_occ[current_device()][occ_kind].load(std::memory_order_relaxed) : 0;
    per_sm = occ > 0 ? occ : 3;
  }
  const int blocks = L.sm_count * per_sm;
  const int needed = (n_items + wpb - 1) / wpb;
  return blocks < needed ? blocks : (needed > 0 ? needed : 1);
}

cudaError_t launch_background(const Launch& L, const PlanView& v) {
  if (v.n_items == 0) return cudaSuccess;
  background_kernel<<<grid_for(L, v.n_items, kWpb, kOccBackground), kWpb * 32, smem_bytes(kWpb), L.stream>>>(
      v, L.n_exp, L.n_dev);
  return cudaGetLastError();
}

// The work queue pays when a launch has many items per warp (its claims
// then balance the warps' finishing times); with few, the grid-stride form
// (fewer registers, no claims) is faster.
constexpr int kQueueItemsPerWarp = 8;
static bool use_queue(const PlanView& v, int blocks) {
  return v.work_ctr && v.n_items >= kQueueItemsPerWarp * kWpb * blocks;
}

cudaError_t launch_pixels_derivs(const Launch& L, const PlanView& v) {
  if (v.n_items == 0) return cudaSuccess;
  if (cudaError_t e = derivs_attr()) return e;
  const int gq = grid_for(L, v.n_items, kWpb, kOccDerivsQ);
  if (use_queue(v, gq))
    derivs_kernel<true><<<gq, kWpb * 32, smem_bytes_derivs(kWpb), L.stream>>>(v, L.n_exp, L.n_dev);
  else
    derivs_kernel<false><<<grid_for(L, v.n_items, kWpb, kOccDerivs), kWpb * 32,
                           smem_bytes_derivs(kWpb), L.stream>>>(v, L.n_exp, L.n_dev);
  return cudaGetLastError();
}

cudaError_t launch_pixels_grad(const Launch& L, const PlanView& v) {
  if (v.n_items == 0) return cudaSuccess;
  const int gq = grid_for(L, v.n_items, kWpb, kOccGradQ);
  if (use_queue(v, gq))
    grad_kernel<true><<<gq, kWpb * 32, smem_bytes_grad(kWpb), L.stream>>>(v, L.n_exp, L.n_dev);
  else
    grad_kernel<false><<<grid_for(L, v.n_items, kWpb, kOccGrad), kWpb * 32, smem_bytes_grad(kWpb),
                         L.stream>>>(v, L.n_exp, L.n_dev);
  return cudaGetLastError();
}

cudaError_t launch_pixels_value(const Launch& L, const PlanView& v, bool keep_render) {
  if (v.n_items == 0) return cudaSuccess;
  const int mode = !keep_render || !v.cache ? 0 : (v.cache_half ? 2 : 1);
  const int gq = grid_for(L, v.n_items, kWpb, kOccValueQ);
  if (use_queue(v, gq))
    value_kernel<true><<<gq, kWpb * 32, smem_bytes(kWpb), L.stream>>>(v, L.n_exp, L.n_dev, mode);
  else
    value_kernel<false><<<grid_for(L, v.n_items, kWpb, kOccValue), kWpb * 32, smem_bytes(kWpb),
                          L.stream>>>(v, L.n_exp, L.n_dev, mode);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const Launch& L, const PlanView& v, const ModelDev* model,
                           const int32_t* status, int n_setup, bool background) {
  const int units = (v.n + 31) / 32 + n_setup + (background ? v.n_items : 0);
  if (units == 0) return cudaSuccess;
  prepare_kernel<<<grid_for(L, units, kWpb, kOccPrepare), kWpb * 32, smem_bytes(kWpb),
                   L.stream>>>(v, model, status, n_setup, background ? 1 : 0, L.n_exp, L.n_dev);
  return cudaGetLastError();
}

cudaError_t launch_commit_render(const Launch& L, const PlanView& v, const int32_t* status) {
  if (v.n_items == 0 || !v.cache || !v.trial_render) return cudaSuccess;
  commit_render_kernel<<<grid_for(L, v.n_items, kWpb, kOccCommit), kWpb * 32, 0, L.stream>>>(
      v, status);
  return cudaGetLastError();
}

cudaError_t launch_render(const Launch& L, const PlanView& v, float* E_out, float* V_out,
                          const celeste_patch* patches) {
  if (v.n_items == 0) return cudaSuccess;
  render_kernel<<<grid_for(L, v.n_items, kWpb), kWpb * 32, smem_bytes(kWpb), L.stream>>>(
      v, L.n_exp, L.n_dev, E_out, V_out, patches);
  return cudaGetLastError();
}

cudaError_t launch_render_cache(const Launch& L, const PlanView& v, const int32_t* status) {
  if (v.n_items == 0 || !v.cache) return cudaSuccess;
  render_cache_kernel<<<grid_for(L, v.n_items, kWpb, kOccRender), kWpb * 32, smem_bytes(kWpb), L.stream>>>(
      v, L.n_exp, L.n_dev, status);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const Launch& L, const PlanView& v, float* Eimg, float* Vimg) {
  if (v.n_items == 0) return cudaSuccess;
  accumulate_kernel<<<grid_for(L, v.n_items, kWpb, kOccRender), kWpb * 32, smem_bytes(kWpb),
                      L.stream>>>(v, L.n_exp, L.n_dev, Eimg, Vimg);
  return cudaGetLastError();
}

cudaError_t launch_field_terms(const Launch& L, const celeste_image* images, int n_images,
                               int blocks_per_image, const float* pixels, const float* sky,
                               const float* Eimg, const float* Vimg, unsigned int* err,
                               double* parts) {
  if (n_images == 0) return cudaSuccess;
  field_term_kernel<<<dim3(blocks_per_image, n_images), 256, 0, L.stream>>>(images, pixels, sky,
                                                                            Eimg, Vimg, err, parts);
  return cudaGetLastError();
}

cudaError_t launch_field_sum(const Launch& L, const double* parts, int n_parts, const double* kl,
                             int n_kl, double* out) {
  field_sum_kernel<<<1, 256, 0, L.stream>>>(parts, n_parts, kl, n_kl, out);
  return cudaGetLastError();
}

cudaError_t launch_background_out(const Launch& L, const PlanView& v, float* bgE, float* bgV,
                                  const celeste_patch* patches) {
  if (v.n_items == 0) return cudaSuccess;
  bg_scatter_kernel<<<grid_for(L, v.n_items, kWpb), kWpb * 32, 0, L.stream>>>(v, bgE, bgV,
                                                                              patches);
  return cudaGetLastError();
}

}  // namespace celeste
