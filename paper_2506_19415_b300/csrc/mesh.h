// The mesh proxy of Sec. 3.1 (Mesh Extraction) and the page assignment of
// Sec. 3.2 (Page Assignment): device kernels for the occupancy of the scene
// slices, the closing and the surface cells (k_mesh.cu), host code for the
// vertex numbering, the quadric simplification, the nearest-triangle
// assignment with subdivision and the page merging (mesh_proxy.cpp).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace vm {

struct MeshGrid {
  double lo[3];
  double h;
  int64_t n[3];  // sample points per axis (voxel centres lo + (i + 1/2) h)
};

// Occupancy of the grid's sample points by the kappa-sigma ellipsoids of the
// Gaussians of opacity >= op_min (decoded arrays, device copies made here),
// closed with the cube of radius `closing`; returns the closed occupancy as
// bytes [nz][ny][nx] (host) and the raw occupancy when raw is not null.
// False with a message on a CUDA failure.
bool mesh_occupancy(const MeshGrid &g, int64_t n, const float *pos, const float *scale, const float *rot,
                    const float *opac, float kappa, double op_min, int closing, std::vector<uint8_t> &closed,
                    std::vector<uint8_t> *raw, std::string &err);

// The surface of a closed occupancy, cube by cube (Kuhn tetrahedra): vertex
// lattice coordinates D (doubled; world lo + D h / 2) in ascending (Dz, Dy,
// Dx) order and triangles in cube order, computed on the device.
bool mesh_surface(const MeshGrid &g, const std::vector<uint8_t> &closed, std::vector<int32_t> &D,
                  std::vector<int32_t> &tris, std::string &err);

// Quadric-error simplification to at most `target` triangles (FP64).
void qem_simplify(std::vector<double> &verts, std::vector<int32_t> &tris, int64_t target);

// Page assignment by nearest triangle with subdivision and greedy merging.
// Inputs: n means (FP32 xyz), the mesh.  Outputs: the subdivided mesh,
// face_page (-1: no page), the means' order in pages with the pages' counts,
// and per page its parent (-1, or for the extra pages of a triangle that
// splitting could not bring within page_size, the page the triangle carries).
void assign_pages(int64_t n, const float *mu, int64_t page_size, std::vector<double> &verts,
                  std::vector<int32_t> &tris, std::vector<int32_t> &face_page, std::vector<int64_t> &order,
                  std::vector<int64_t> &counts, std::vector<int64_t> &parent);

// Nearest triangle (FP64 distance, ties to the lower index) of each point.
struct TriIndex;
TriIndex *tri_index_build(const std::vector<double> &verts, const std::vector<int32_t> &tris);
int32_t tri_index_nearest(const TriIndex *ix, const double p[3]);
void tri_index_free(TriIndex *ix);

}  // namespace vm
