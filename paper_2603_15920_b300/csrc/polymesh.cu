// Geometry of a polyhedral mesh given by vertices and face vertex loops (the
// form of an OpenFOAM polyMesh), so that meshes made elsewhere can feed the
// static graph arrays of Sec. 2.4.1 (S_f, x_f, V_i, C_i).  Host code, run once
// per mesh before difvm_mesh_create.
//
// Faces: a loop of n >= 3 vertices is split into n triangles around the loop's
// vertex average; the area vector is the sum of the triangles' area vectors and
// the centroid their centroids weighted by the triangles' signed areas along
// the face normal.  Cells: each face with the average of the cell's face
// centroids forms a pyramid; the volume is the sum of the pyramids' signed
// volumes and the centroid their centroids (3/4 of the way from the apex to
// the base centroid) weighted by volume.  Both decompositions are exact for
// planar faces, convex or not; a warped face gets the triangle-fan
// approximation.
#include <cmath>
#include <vector>

#include "difvm_internal.cuh"

namespace difvm {
namespace {

struct P3 {
  double x, y, z;
};
inline P3 operator+(P3 a, P3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline P3 operator-(P3 a, P3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline P3 operator*(double s, P3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(P3 a, P3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline P3 cross(P3 a, P3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

}  // namespace
}  // namespace difvm

using difvm::P3;

extern "C" difvm_status difvm_polymesh_geometry(int32_t n_points, const double* points, int32_t n_faces,
                                                const int32_t* face_ptr, const int32_t* face_pts,
                                                int32_t n_cells, const int32_t* owner, int32_t n_internal,
                                                const int32_t* neighbour, double* Sf, double* Cf, double* V,
                                                double* C) {
  using namespace difvm;
  if (n_points < 4 || n_faces < 4 || n_cells < 1 || n_internal < 0 || n_internal > n_faces)
    return set_error(DIFVM_EINVAL, "polymesh: bad sizes (points %d, faces %d, cells %d, internal %d)", n_points,
                     n_faces, n_cells, n_internal);
  if (!points || !face_ptr || !face_pts || !owner || (n_internal > 0 && !neighbour) || !Sf || !Cf || !V || !C)
    return set_error(DIFVM_EINVAL, "polymesh: null array");
  if (face_ptr[0] != 0) return set_error(DIFVM_EINVAL, "polymesh: face_ptr[0] != 0");
  auto pt = [&](int v) { return P3{points[3 * v], points[3 * v + 1], points[3 * v + 2]}; };
  // faces
  for (int f = 0; f < n_faces; ++f) {
    const int a = face_ptr[f], b = face_ptr[f + 1];
    if (b - a < 3) return set_error(DIFVM_EINVAL, "polymesh: face %d has %d vertices", f, b - a);
    for (int k = a; k < b; ++k)
      if (face_pts[k] < 0 || face_pts[k] >= n_points)
        return set_error(DIFVM_EINVAL, "polymesh: face %d vertex %d out of range", f, face_pts[k]);
    if (owner[f] < 0 || owner[f] >= n_cells) return set_error(DIFVM_EINVAL, "polymesh: owner[%d] out of range", f);
    if (f < n_internal && (neighbour[f] < 0 || neighbour[f] >= n_cells || neighbour[f] == owner[f]))
      return set_error(DIFVM_EINVAL, "polymesh: neighbour[%d] out of range or equal to the owner", f);
    P3 avg{0, 0, 0};
    for (int k = a; k < b; ++k) avg = avg + pt(face_pts[k]);
    avg = (1.0 / (b - a)) * avg;
    P3 S{0, 0, 0};
    for (int k = a; k < b; ++k) {
      const P3 p0 = pt(face_pts[k]), p1 = pt(face_pts[k + 1 < b ? k + 1 : a]);
      S = S + 0.5 * cross(p1 - p0, avg - p0);
    }
    const double smag = std::sqrt(dot(S, S));
    if (!(smag > 0)) return set_error(DIFVM_EINVAL, "polymesh: face %d has zero area", f);
    // centroid: triangle centroids weighted by their signed areas along the
    // face normal (exact also for non-convex planar faces)
    const P3 nh = (1.0 / smag) * S;
    P3 ac{0, 0, 0};
    double asum = 0.0;
    for (int k = a; k < b; ++k) {
      const P3 p0 = pt(face_pts[k]), p1 = pt(face_pts[k + 1 < b ? k + 1 : a]);
      const double ar = 0.5 * dot(cross(p1 - p0, avg - p0), nh);
      asum += ar;
      ac = ac + (ar / 3.0) * (p0 + p1 + avg);
    }
    const P3 xf = (1.0 / asum) * ac;
    Sf[3 * f] = S.x; Sf[3 * f + 1] = S.y; Sf[3 * f + 2] = S.z;
    Cf[3 * f] = xf.x; Cf[3 * f + 1] = xf.y; Cf[3 * f + 2] = xf.z;
  }
  // cells: apex = average of the face centroids
  std::vector<P3> apex(n_cells, P3{0, 0, 0});
  std::vector<int> nfc(n_cells, 0);
  auto xf = [&](int f) { return P3{Cf[3 * f], Cf[3 * f + 1], Cf[3 * f + 2]}; };
  auto sf = [&](int f) { return P3{Sf[3 * f], Sf[3 * f + 1], Sf[3 * f + 2]}; };
  for (int f = 0; f < n_faces; ++f) {
    apex[owner[f]] = apex[owner[f]] + xf(f);
    nfc[owner[f]]++;
    if (f < n_internal) {
      apex[neighbour[f]] = apex[neighbour[f]] + xf(f);
      nfc[neighbour[f]]++;
    }
  }
  for (int i = 0; i < n_cells; ++i) {
    if (nfc[i] < 4) return set_error(DIFVM_EINVAL, "polymesh: cell %d has %d faces", i, nfc[i]);
    apex[i] = (1.0 / nfc[i]) * apex[i];
  }
  std::vector<double> vol(n_cells, 0.0);
  std::vector<P3> mom(n_cells, P3{0, 0, 0});
  auto pyramid = [&](int i, int f, double sign) {
    const double v = sign * dot(sf(f), xf(f) - apex[i]) / 3.0;
    vol[i] += v;
    mom[i] = mom[i] + v * (0.75 * xf(f) + 0.25 * apex[i]);
  };
  for (int f = 0; f < n_faces; ++f) {
    pyramid(owner[f], f, 1.0);
    if (f < n_internal) pyramid(neighbour[f], f, -1.0);
  }
  for (int i = 0; i < n_cells; ++i) {
    if (!(vol[i] > 0))
      return set_error(DIFVM_EINVAL, "polymesh: cell %d has volume %g (faces not oriented out of the owner?)", i,
                       vol[i]);
    const P3 c = (1.0 / vol[i]) * mom[i];
    V[i] = vol[i];
    C[3 * i] = c.x; C[3 * i + 1] = c.y; C[3 * i + 2] = c.z;
  }
  return DIFVM_OK;
}
