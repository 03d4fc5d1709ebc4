// Device part of the mesh proxy (Sec. 3.1, Mesh Extraction):
//   occupancy  a thread per Gaussian marks the grid's sample points (voxel
//              centres) inside its kappa-sigma ellipsoid.  The paper draws
//              each ellipsoid's section with every scene slice (the ellipse
//              of Hartmann's construction); marking the sample points of a
//              slice inside that ellipse is the same as testing each point of
//              a box around the ellipsoid against the ellipsoid, which is
//              what the kernel does, with one FP32 formula in a fixed order
//              (this file is compiled with -fmad=false): d = x - mu,
//              w_j = (R_0j d_0 + R_1j d_1) + R_2j d_2, u_j = w_j / s_j,
//              (u_0^2 + u_1^2) + u_2^2 <= kappa^2.
//   closing    dilation then erosion with the cube of radius r, separable
//              per axis, on the grid padded by r empty layers (the closing of
//              the set in unbounded empty space).
//   surface    per cube of 8 neighbouring sample points (grid padded by one
//              empty layer): its inside pattern picks, from a table generated
//              on the host by cutting the cube into the 6 tetrahedra around
//              its main diagonal, triangles whose vertices are midpoints of
//              inside-outside edges, oriented from inside to outside; a count
//              pass, a host scan, then an emission pass in cube order.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "mesh.h"

namespace vm {
namespace {

constexpr int kMaxCubeTris = 12;  // 6 tetrahedra x at most 2 triangles
struct CaseTable {
  uint8_t count[256];
  uint8_t edge[256][kMaxCubeTris][3][2];  // (inside corner, outside corner) per triangle vertex
};
__constant__ CaseTable c_table;

const int kCorner[8][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 0}, {0, 0, 1}, {1, 0, 1}, {0, 1, 1}, {1, 1, 1}};

// the table: tetrahedra 0 -> e_a -> e_a + e_b -> 7 for the axis orders
// (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y), (z,y,x)
void make_table(CaseTable &t) {
  static const int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  std::memset(&t, 0, sizeof(t));
  for (int cs = 0; cs < 256; ++cs) {
    int nt = 0;
    for (int k = 0; k < 6; ++k) {
      const int c1 = 1 << perms[k][0], c2 = c1 | (1 << perms[k][1]);
      const int tet[4] = {0, c1, c2, 7};
      int ins[4], outs[4], ni = 0, no = 0;
      for (int v = 0; v < 4; ++v) {
        if ((cs >> tet[v]) & 1) ins[ni++] = v;
        else outs[no++] = v;
      }
      int tri[2][3][2], ntri = 0;
      if (ni == 1) {
        for (int j = 0; j < 3; ++j) { tri[0][j][0] = ins[0]; tri[0][j][1] = outs[j]; }
        ntri = 1;
      } else if (ni == 3) {
        for (int j = 0; j < 3; ++j) { tri[0][j][0] = ins[j]; tri[0][j][1] = outs[0]; }
        ntri = 1;
      } else if (ni == 2) {
        const int a0 = ins[0], a1 = ins[1], b0 = outs[0], b1 = outs[1];
        const int q[2][3][2] = {{{a0, b0}, {a0, b1}, {a1, b1}}, {{a0, b0}, {a1, b1}, {a1, b0}}};
        std::memcpy(tri, q, sizeof(q));
        ntri = 2;
      }
      for (int r = 0; r < ntri; ++r) {
        int e[3][2];
        for (int j = 0; j < 3; ++j) { e[j][0] = tet[tri[r][j][0]]; e[j][1] = tet[tri[r][j][1]]; }
        // orientation from inside to outside, on doubled coordinates
        long long v[3][3];
        for (int j = 0; j < 3; ++j)
          for (int a = 0; a < 3; ++a)
            v[j][a] = ((2 * kCorner[e[j][0]][a] + 1) + (2 * kCorner[e[j][1]][a] + 1)) / 2;
        const long long u1[3] = {v[1][0] - v[0][0], v[1][1] - v[0][1], v[1][2] - v[0][2]};
        const long long u2[3] = {v[2][0] - v[0][0], v[2][1] - v[0][1], v[2][2] - v[0][2]};
        const long long nrm[3] = {u1[1] * u2[2] - u1[2] * u2[1], u1[2] * u2[0] - u1[0] * u2[2],
                                  u1[0] * u2[1] - u1[1] * u2[0]};
        long long dot = 0;
        for (int a = 0; a < 3; ++a) dot += nrm[a] * (kCorner[e[0][1]][a] - kCorner[e[0][0]][a]);
        if (dot < 0) {
          std::swap(e[1][0], e[2][0]);
          std::swap(e[1][1], e[2][1]);
        }
        for (int j = 0; j < 3; ++j) {
          t.edge[cs][nt][j][0] = (uint8_t)e[j][0];
          t.edge[cs][nt][j][1] = (uint8_t)e[j][1];
        }
        ++nt;
      }
    }
    t.count[cs] = (uint8_t)nt;
  }
}

__global__ void occupancy_kernel(int64_t n, const float *pos, const float *scale, const float *rot, const float *opac,
                                 float lo0, float lo1, float lo2, float h, int nx, int ny, int nz, float kappa,
                                 double op_min, uint8_t *occ) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || !(opac[i] >= (float)op_min)) return;
  const float w = rot[4 * i], x = rot[4 * i + 1], y = rot[4 * i + 2], z = rot[4 * i + 3];
  const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z, wx = w * x, wy = w * y,
              wz = w * z;
  float R[3][3];
  R[0][0] = 1.0f - 2.0f * (yy + zz); R[0][1] = 2.0f * (xy - wz); R[0][2] = 2.0f * (xz + wy);
  R[1][0] = 2.0f * (xy + wz); R[1][1] = 1.0f - 2.0f * (xx + zz); R[1][2] = 2.0f * (yz - wx);
  R[2][0] = 2.0f * (xz - wy); R[2][1] = 2.0f * (yz + wx); R[2][2] = 1.0f - 2.0f * (xx + yy);
  const float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
  const float mu[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};
  const float lo[3] = {lo0, lo1, lo2};
  const int dims[3] = {nx, ny, nz};
  // a box holding every sample point the FP32 test can accept (1% margin)
  int i0[3], i1[3];
  for (int a = 0; a < 3; ++a) {
    double sa = 0.0;
    for (int k = 0; k < 3; ++k) sa += (double)R[a][k] * R[a][k] * (double)s[k] * s[k];
    const double ext = (double)kappa * sqrt(sa) * 1.01 + 1e-5;
    const double c0 = floor(((double)mu[a] - ext - (double)lo[a]) / (double)h - 0.5);
    const double c1 = ceil(((double)mu[a] + ext - (double)lo[a]) / (double)h - 0.5);
    i0[a] = (int)fmax(c0, 0.0);
    i1[a] = (int)fmin(c1, (double)(dims[a] - 1));
    if (i1[a] < i0[a]) return;
  }
  const float k2 = kappa * kappa;
  for (int iz = i0[2]; iz <= i1[2]; ++iz)
    for (int iy = i0[1]; iy <= i1[1]; ++iy)
      for (int ix = i0[0]; ix <= i1[0]; ++ix) {
        const int c[3] = {ix, iy, iz};
        float d[3];
        for (int a = 0; a < 3; ++a) d[a] = (lo[a] + ((float)c[a] + 0.5f) * h) - mu[a];
        float q = 0.0f;
        float u[3];
        for (int j = 0; j < 3; ++j) u[j] = ((R[0][j] * d[0] + R[1][j] * d[1]) + R[2][j] * d[2]) / s[j];
        q = (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2];
        if (q <= k2) occ[((int64_t)iz * ny + iy) * nx + ix] = 1;
      }
}

// one separable pass of a cube filter along axis a on a [nz][ny][nx] byte grid:
// out = OR (dilate) or AND (erode) over the window of radius r, outside empty
__global__ void box_pass_kernel(const uint8_t *in, uint8_t *out, int nx, int ny, int nz, int a, int r, int dilate) {
  const int64_t total = (int64_t)nx * ny * nz;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((int64_t)nx * ny));
    const int c = a == 0 ? x : (a == 1 ? y : z), n = a == 0 ? nx : (a == 1 ? ny : nz);
    const int64_t stride = a == 0 ? 1 : (a == 1 ? nx : (int64_t)nx * ny);
    uint8_t acc = dilate ? 0 : 1;
    for (int k = -r; k <= r; ++k) {
      const int cc = c + k;
      const uint8_t val = (cc < 0 || cc >= n) ? 0 : in[v + (int64_t)k * stride];
      acc = dilate ? (acc | val) : (acc & val);
    }
    out[v] = acc;
  }
}

__device__ __forceinline__ uint8_t sample_at(const uint8_t *g, int nx, int ny, int nz, int x, int y, int z) {
  if (x < 0 || y < 0 || z < 0 || x >= nx || y >= ny || z >= nz) return 0;
  return g[((int64_t)z * ny + y) * nx + x];
}

// cube (x, y, z) of the padded grid: corner c at sample (x - 1 + cx, ...)
__device__ __forceinline__ int cube_case(const uint8_t *g, int nx, int ny, int nz, int x, int y, int z) {
  int cs = 0;
  for (int c = 0; c < 8; ++c)
    cs |= sample_at(g, nx, ny, nz, x - 1 + (c & 1), y - 1 + ((c >> 1) & 1), z - 1 + ((c >> 2) & 1)) << c;
  return cs;
}

__global__ void cube_count_kernel(const uint8_t *g, int nx, int ny, int nz, uint8_t *cnt) {
  const int64_t total = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % (nx + 1)), y = (int)((v / (nx + 1)) % (ny + 1)), z = (int)(v / ((int64_t)(nx + 1) * (ny + 1)));
    cnt[v] = c_table.count[cube_case(g, nx, ny, nz, x, y, z)];
  }
}

// triangles of each cube at its scanned offset: 9 ints (D of 3 vertices)
__global__ void cube_emit_kernel(const uint8_t *g, int nx, int ny, int nz, const uint32_t *off, int32_t *out) {
  const int64_t total = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < total; v += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(v % (nx + 1)), y = (int)((v / (nx + 1)) % (ny + 1)), z = (int)(v / ((int64_t)(nx + 1) * (ny + 1)));
    const int cs = cube_case(g, nx, ny, nz, x, y, z);
    const int nt = c_table.count[cs];
    const int base[3] = {x - 1, y - 1, z - 1};
    for (int t = 0; t < nt; ++t)
      for (int j = 0; j < 3; ++j) {
        const int a = c_table.edge[cs][t][j][0], b = c_table.edge[cs][t][j][1];
        const int ca[3] = {a & 1, (a >> 1) & 1, (a >> 2) & 1}, cb[3] = {b & 1, (b >> 1) & 1, (b >> 2) & 1};
        for (int k = 0; k < 3; ++k)
          out[((int64_t)off[v] + t) * 9 + 3 * j + k] =
              ((2 * (base[k] + ca[k]) + 1) + (2 * (base[k] + cb[k]) + 1)) / 2;
      }
  }
}

template <class T>
struct DevBuf {
  T *p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
  bool alloc(size_t n) { return cudaMalloc(&p, sizeof(T) * (n ? n : 1)) == cudaSuccess; }
};

bool ok_or(cudaError_t e, const char *what, std::string &err) {
  if (e == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(e);
  return false;
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 148 * 16); }

}  // namespace

bool mesh_occupancy(const MeshGrid &g, int64_t n, const float *pos, const float *scale, const float *rot,
                    const float *opac, float kappa, double op_min, int closing, std::vector<uint8_t> &closed,
                    std::vector<uint8_t> *raw, std::string &err) {
  const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
  const int64_t NV = (int64_t)nx * ny * nz;
  DevBuf<float> dpos, dsc, drot, dop;
  DevBuf<uint8_t> docc;
  if (!(dpos.alloc(3 * n) && dsc.alloc(3 * n) && drot.alloc(4 * n) && dop.alloc(n) && docc.alloc(NV)))
    return ok_or(cudaErrorMemoryAllocation, "mesh occupancy buffers", err);
  if (!ok_or(cudaMemcpy(dpos.p, pos, 12 * n, cudaMemcpyHostToDevice), "copy", err) ||
      !ok_or(cudaMemcpy(dsc.p, scale, 12 * n, cudaMemcpyHostToDevice), "copy", err) ||
      !ok_or(cudaMemcpy(drot.p, rot, 16 * n, cudaMemcpyHostToDevice), "copy", err) ||
      !ok_or(cudaMemcpy(dop.p, opac, 4 * n, cudaMemcpyHostToDevice), "copy", err) ||
      !ok_or(cudaMemset(docc.p, 0, NV), "clear", err))
    return false;
  if (n > 0)
    occupancy_kernel<<<(unsigned)((n + 127) / 128), 128>>>(n, dpos.p, dsc.p, drot.p, dop.p, (float)g.lo[0],
                                                            (float)g.lo[1], (float)g.lo[2], (float)g.h, nx, ny, nz,
                                                            kappa, op_min, docc.p);
  if (!ok_or(cudaGetLastError(), "occupancy kernel", err) || !ok_or(cudaDeviceSynchronize(), "occupancy", err))
    return false;
  if (raw) {
    raw->resize(NV);
    if (!ok_or(cudaMemcpy(raw->data(), docc.p, NV, cudaMemcpyDeviceToHost), "copy back", err)) return false;
  }
  closed.resize(NV);
  if (closing <= 0) return ok_or(cudaMemcpy(closed.data(), docc.p, NV, cudaMemcpyDeviceToHost), "copy back", err);
  // padded by r empty layers
  const int r = closing, px = nx + 2 * r, py = ny + 2 * r, pz = nz + 2 * r;
  const int64_t NP = (int64_t)px * py * pz;
  std::vector<uint8_t> h(NV), hp(NP, 0);
  if (!ok_or(cudaMemcpy(h.data(), docc.p, NV, cudaMemcpyDeviceToHost), "copy back", err)) return false;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      std::memcpy(&hp[(((int64_t)(z + r) * py) + (y + r)) * px + r], &h[((int64_t)z * ny + y) * nx], nx);
  DevBuf<uint8_t> a, b;
  if (!(a.alloc(NP) && b.alloc(NP))) return ok_or(cudaErrorMemoryAllocation, "closing buffers", err);
  if (!ok_or(cudaMemcpy(a.p, hp.data(), NP, cudaMemcpyHostToDevice), "copy", err)) return false;
  uint8_t *src = a.p, *dst = b.p;
  for (int dil = 1; dil >= 0; --dil)
    for (int ax = 0; ax < 3; ++ax) {
      box_pass_kernel<<<grid_for(NP), 256>>>(src, dst, px, py, pz, ax, r, dil);
      std::swap(src, dst);
    }
  if (!ok_or(cudaGetLastError(), "closing kernel", err) ||
      !ok_or(cudaMemcpy(hp.data(), src, NP, cudaMemcpyDeviceToHost), "copy back", err))
    return false;
  for (int z = 0; z < nz; ++z)
    for (int y = 0; y < ny; ++y)
      std::memcpy(&closed[((int64_t)z * ny + y) * nx], &hp[(((int64_t)(z + r) * py) + (y + r)) * px + r], nx);
  return true;
}

bool mesh_surface(const MeshGrid &g, const std::vector<uint8_t> &closed, std::vector<int32_t> &D,
                  std::vector<int32_t> &tris, std::string &err) {
  // (built once, thread-safely, on first use)
  static const CaseTable table = [] {
    CaseTable t;
    make_table(t);
    return t;
  }();
  if (!ok_or(cudaMemcpyToSymbol(c_table, &table, sizeof(table)), "case table", err)) return false;
  const int nx = (int)g.n[0], ny = (int)g.n[1], nz = (int)g.n[2];
  const int64_t NV = (int64_t)nx * ny * nz, NC = (int64_t)(nx + 1) * (ny + 1) * (nz + 1);
  DevBuf<uint8_t> dg, dcnt;
  DevBuf<uint32_t> doff;
  if (!(dg.alloc(NV) && dcnt.alloc(NC) && doff.alloc(NC))) return ok_or(cudaErrorMemoryAllocation, "surface", err);
  if (!ok_or(cudaMemcpy(dg.p, closed.data(), NV, cudaMemcpyHostToDevice), "copy", err)) return false;
  cube_count_kernel<<<grid_for(NC), 256>>>(dg.p, nx, ny, nz, dcnt.p);
  std::vector<uint8_t> cnt(NC);
  if (!ok_or(cudaGetLastError(), "count kernel", err) ||
      !ok_or(cudaMemcpy(cnt.data(), dcnt.p, NC, cudaMemcpyDeviceToHost), "copy back", err))
    return false;
  std::vector<uint32_t> off(NC);
  uint64_t tot = 0;
  for (int64_t c = 0; c < NC; ++c) {
    off[c] = (uint32_t)tot;
    tot += cnt[c];
  }
  if (tot >= (1ull << 31)) { err = "surface has too many triangles"; return false; }
  DevBuf<int32_t> dout;
  if (!dout.alloc(9 * tot)) return ok_or(cudaErrorMemoryAllocation, "surface triangles", err);
  if (!ok_or(cudaMemcpy(doff.p, off.data(), 4 * NC, cudaMemcpyHostToDevice), "copy", err)) return false;
  cube_emit_kernel<<<grid_for(NC), 256>>>(dg.p, nx, ny, nz, doff.p, dout.p);
  std::vector<int32_t> tv(9 * tot);
  if (!ok_or(cudaGetLastError(), "emit kernel", err) ||
      !ok_or(cudaMemcpy(tv.data(), dout.p, 4 * tv.size(), cudaMemcpyDeviceToHost), "copy back", err))
    return false;
  // vertices numbered in ascending (Dz, Dy, Dx)
  auto key = [](const int32_t *d) {
    return ((uint64_t)(uint32_t)d[2] << 42) | ((uint64_t)(uint32_t)d[1] << 21) | (uint64_t)(uint32_t)d[0];
  };
  std::vector<uint64_t> keys(3 * tot);
  for (uint64_t i = 0; i < 3 * tot; ++i) keys[i] = key(&tv[3 * i]);
  std::vector<uint64_t> u(keys);
  std::sort(u.begin(), u.end());
  u.erase(std::unique(u.begin(), u.end()), u.end());
  D.resize(3 * u.size());
  for (size_t i = 0; i < u.size(); ++i) {
    D[3 * i] = (int32_t)(u[i] & 0x1FFFFF);
    D[3 * i + 1] = (int32_t)((u[i] >> 21) & 0x1FFFFF);
    D[3 * i + 2] = (int32_t)(u[i] >> 42);
  }
  tris.resize(3 * tot);
  for (uint64_t i = 0; i < 3 * tot; ++i)
    tris[i] = (int32_t)(std::lower_bound(u.begin(), u.end(), keys[i]) - u.begin());
  return true;
}

}  // namespace vm
