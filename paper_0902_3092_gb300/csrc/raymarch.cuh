// raymarch.cuh -- the cells a straight ray crosses in the (r, theta) grid and its path length in each,
// from the closed-form crossings of the ray with the radial spheres and the polar cones.
//
// The ray is X(s) = X0 + s o with o = (sin i, 0, cos i) and X0 = p e1 + q e2 = (-q cos i, p, q sin i)
// (sky point (p, q), X0 . o = 0), so r(s)^2 = b^2 + s^2 with b^2 = p^2 + q^2: r falls until s = 0 and
// grows after it, and the next radial face is the inner sphere of the current shell while s < 0 (if
// the ray reaches it) and the outer one otherwise, at s = -+ sqrt(r_f^2 - b^2). The polar angle turns
// at most once: d cos(theta)/ds has the sign of cos(i) b^2 - z0 s (z0 = q sin i), so the next polar
// face is the one on the side theta moves towards, and the turning point s = cos(i) b^2 / z0 is an event
// that changes the side without leaving the cell. A cone theta_f meets the ray where
// A s^2 + 2 B s + C = 0 with A = cos^2 sin^2 i - sin^2 cos^2 i, B = -(cos^2 + sin^2) q sin i cos i,
// C = cos^2 (x0^2 + y0^2) - sin^2 z0^2 (cos, sin of theta_f); a root counts if it lies ahead, on the
// face's nappe (z of the sign of cos theta_f), and is crossed in the direction theta moves. The
// midplane face is the plane z = 0.
//
// Cost: a radial event leaves the next polar crossing valid and a polar event leaves the next radial
// crossing valid, so each step computes one new root (a square root for a sphere, a quadratic for a
// cone, with 1/A per face and inclination from a table). Positions never accumulate: every crossing is
// computed from (X0, o).
#pragma once

#include <cmath>

#if defined(__CUDACC__)
#define MCRT_HD __host__ __device__ __forceinline__
#else
#define MCRT_HD inline
#endif

namespace mcrt {

// Per polar face and inclination: the quadratic's A, its reciprocal (infinity for A = 0), cos^2 + sin^2,
// cos^2, sin^2 and the face kind (+1 cone above the midplane, -1 below, 0 the midplane plane, 2 the axis).
template <class R>
struct FaceCoef {
  R A, iA, cs, c2, s2;
  int kind;
};

template <class R>
MCRT_HD FaceCoef<R> face_coef(R c2, R s2, int kind, R si, R ci) {
  FaceCoef<R> f;
  f.A = c2 * si * si - s2 * ci * ci;
  f.iA = f.A != (R)0 ? (R)1 / f.A : (R)INFINITY;
  f.cs = c2 + s2;
  f.c2 = c2;
  f.s2 = s2;
  f.kind = kind;
  return f;
}

template <class R>
struct RayGrid {
  int nr, nt;
  const R* rf2;             // nr+1 squared radial faces
  const R* cf;              // nt+1 cos theta_f (decreasing)
  const FaceCoef<R>* face;  // nt+1 face coefficients for the inclination of the rays
};

// Polar cell of direction cos(theta) = mu: the last face k in 0..nt-1 with cos theta_k >= mu.
template <class R>
MCRT_HD int polar_index(const RayGrid<R>& G, R mu) {
  int lo = 0, hi = G.nt;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (G.cf[mid] >= mu) lo = mid; else hi = mid;
  }
  return lo;
}

// Calls emit(ir, it, L) for every cell the ray through sky point (p, q) crosses, in order of increasing
// s (towards the observer), L the path length in the grid's length unit. (si, ci) = (sin i, cos i) of
// the inclination the face table was built for. Returns the number of events, 0 if the ray misses the
// grid, -1 if it took more than max_events.
template <class R, class Emit>
MCRT_HD int march_ray(const RayGrid<R>& G, R p, R q, R si, R ci, int max_events, Emit&& emit) {
  using std::sqrt;
  const R inf = (R)INFINITY;
  const R b2 = p * p + q * q;
  if (!(b2 < G.rf2[G.nr])) return 0;
  const R z0 = q * si;
  const R P1 = q * q * ci * ci + p * p;  // x0^2 + y0^2
  const R P2 = z0 * z0;
  const R Bq = -q * si * ci;
  const R cb2 = ci * b2;
  R s = -sqrt(G.rf2[G.nr] - b2);
  R s0 = s;  // where the ray entered the current cell
  int ir = G.nr - 1;
  int it = polar_index(G, (z0 + s * ci) / sqrt(b2 + s * s));
  // the polar angle falls (down) before the turning point s_e = cos(i) b^2 / z0 when z0 > 0 and after
  // it when z0 < 0; the side is decided here and flipped at the turning point, never re-derived from
  // the sign of cos(i) b^2 - z0 s near it, where rounding decides that sign
  R se = inf;
  bool turn = false, down;
  if (z0 != (R)0) {
    se = cb2 / z0;
    turn = se > s;
    down = turn ? z0 > (R)0 : z0 < (R)0;
  } else {
    down = cb2 > (R)0;
  }
  R sr = inf, st = inf;
  int dr = 1;
  bool need_r = true, need_t = true;
  for (int n = 1; n <= max_events; ++n) {
    if (need_r) {  // radial face ahead
      if (s < (R)0 && G.rf2[ir] > b2) {
        sr = -sqrt(G.rf2[ir] - b2);
        dr = -1;
      } else {
        sr = sqrt(G.rf2[ir + 1] - b2);
        dr = 1;
      }
      need_r = false;
    }
    if (need_t) {  // polar face on the side theta moves towards
      const FaceCoef<R> F = G.face[down ? it : it + 1];
      st = inf;
      if (F.kind == 0) {
        if (ci != (R)0) {
          const R sp = -z0 / ci;
          if (sp >= s) st = sp;
        }
      } else if (F.kind != 2) {
        const R B = F.cs * Bq;
        const R C = F.c2 * P1 - F.s2 * P2;
        const R disc = B * B - F.A * C;
        if (disc >= (R)0) {
          const R h = -(B + copysign(sqrt(disc), B));
          const R r1 = h * F.iA;
          const R r2 = h != (R)0 ? C / h : inf;
          const R sg = (R)F.kind;
          // ahead, on the face's nappe, crossed in the direction theta moves
          const bool ok1 = r1 >= s && sg * (z0 + r1 * ci) >= (R)0 && (down ? cb2 - z0 * r1 >= (R)0 : cb2 - z0 * r1 <= (R)0);
          const bool ok2 = r2 >= s && sg * (z0 + r2 * ci) >= (R)0 && (down ? cb2 - z0 * r2 >= (R)0 : cb2 - z0 * r2 <= (R)0);
          if (ok1) st = r1;
          if (ok2 && r2 < st) st = r2;
        }
      }
      need_t = false;
    }
    // turning point of theta inside the cell
    const R sx = turn ? se : inf;
    if (sx < st && sx < sr) {
      s = sx > s ? sx : s;
      turn = false;
      down = !down;
      need_t = true;
      continue;
    }
    if (st < sr) {
      const R e = st > s ? st : s;
      emit(ir, it, e - s0);
      s = s0 = e;
      it += down ? -1 : 1;
      need_t = true;
    } else {
      const R e = sr > s ? sr : s;
      emit(ir, it, e - s0);
      s = s0 = e;
      ir += dr;
      need_r = true;
      if (ir >= G.nr) return n;
      if (ir < 0) {  // the cavity inside the inner radius: no dust, out at the far side of r_in
        s = s0 = sqrt(G.rf2[0] - b2);
        ir = 0;
        it = polar_index(G, (z0 + s * ci) / sqrt(b2 + s * s));
        need_t = true;
      }
    }
  }
  return -1;
}

}  // namespace mcrt
