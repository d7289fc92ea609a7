// A mesh split into (x, y) pencils of elements: the domain decomposition of
// Sec. 3.1 (the element loop distributed over partitions, with the face data
// neighbours need exchanged between them), in its single-GPU form.
//
// Each partition is a handle of its own (create_handle with a PartSpec): its
// interior elements plus one ghost element on each side in x and y.  The DG
// kernels read a neighbour's face nodes through the storage index of the
// neighbouring element, so on a partition boundary they read the ghost
// element, whose face nodes the halo exchange has filled.  Two exchanges per
// stage, as the two passes need them:
//   A, before the gradient pass: the state (FP64 Q, or the FP32 shadow S) and
//      its four thermodynamic fields at the face nodes; the flux pass reads
//      the same (the state does not change between the two passes);
//   B, before the flux pass: the five F2 components of the face's direction.
// An exchange is a pack kernel per partition and side (gather of the face
// nodes into a contiguous send buffer), one copy per side into the receiving
// partition's buffer (device to device on this GPU; the step a multi-GPU run
// makes with a point-to-point send/receive), and an unpack kernel (scatter
// into the ghost element).  The halo plan (which face nodes, in which order)
// is the host function halo_plan, also exported as cmles_halo_plan.
//
// The result is bit-identical to the whole mesh's: every element runs the
// same kernel code on the same values.  Budgets are summed over partitions
// on the host (the allreduce of a multi-GPU run), so they agree to rounding.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "handle.h"

using namespace cmles_host;

struct cmles_group_t {
  cmles_mesh mesh;
  cmles_params prm;
  int px = 1, py = 1;
  std::vector<cmles_handle> part;
  std::vector<cmles_host::PartSpec> spec;
  // per partition and side: neighbour partition, face-node count, device
  // index lists (storage node index e Np + n) and send / receive buffers
  struct Side {
    int nb = -1;
    long long count = 0;
    long long *send_idx = nullptr, *recv_idx = nullptr;
    void *send_buf = nullptr, *recv_buf = nullptr;
  };
  std::vector<Side> side;  // [partition][4]
  // FP32 partitions: FP64 scratch for the tendency's input and output
  std::vector<double *> tmpQ, tmpR;
  cudaStream_t stream = 0;
  std::string err;
  long long halo_bytes_stage = 0;
};

namespace {

cmles_status gfail(cmles_group g, cmles_status st, const std::string &msg) {
  if (g) g->err = msg;
  return st;
}

#define GCK(call)                                                                            \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return gfail(g, CMLES_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// part idx of n elements split into `parts` nearly equal runs
void split(int n, int parts, int idx, int *start, int *len) {
  const int base = n / parts, extra = n % parts;
  *start = idx * base + std::min(idx, extra);
  *len = base + (idx < extra ? 1 : 0);
}

// Local storage element of interior coordinates (ex, ey, ez) of a partition
// with nx x ny interior columns (-1 and nx / ny are the ghosts).
long long storage_elem(int nx, int ny, int ex, int ey, int ez) {
  return (ex + 1) + (long long)(nx + 2) * ((ey + 1) + (long long)(ny + 2) * ez);
}

// The halo plan of partition `rank`.  Side s = 0 -x, 1 +x, 2 -y, 3 +y.
// send[s]: the face nodes of the partition's elements on side s, for the
// neighbour across s; recv[s]: the face nodes of the ghost elements on side
// s that the neighbour's send[s ^ 1] fills, entry for entry.  Entries are
// ordered by element layer ez, then the element's position along the side,
// then the face node (t1 + Nq t2, t1 and t2 the two in-face indices in
// x, y, z order); each is a storage node index e Np + n.
bool halo_plan(const cmles_mesh &m, int px, int py, int rank, int nb[4], std::vector<long long> send[4],
               std::vector<long long> recv[4]) {
  if (px < 1 || py < 1 || rank < 0 || rank >= px * py || px > m.nex || py > m.ney) return false;
  const int N = m.N, Nq = N + 1, Np = Nq * Nq * Nq;
  const int ix = rank % px, iy = rank / px;
  int x0, nx, y0, ny;
  split(m.nex, px, ix, &x0, &nx);
  split(m.ney, py, iy, &y0, &ny);
  for (int s = 0; s < 4; ++s) {
    const int d = s >> 1, hi = s & 1;
    const int np = d == 0 ? px : py, i = d == 0 ? ix : iy;
    int j = i + (hi ? 1 : -1);
    if (j < 0 || j >= np) j = m.periodic[d] ? (j + np) % np : -1;
    nb[s] = j < 0 ? -1 : (d == 0 ? j + px * iy : ix + px * j);
    send[s].clear();
    recv[s].clear();
    if (nb[s] < 0) continue;
    const int along = d == 0 ? ny : nx;
    const int a = hi ? N : 0;  // this side's face of an element, in its own index
    for (int ez = 0; ez < m.nez; ++ez)
      for (int p = 0; p < along; ++p) {
        const int bex = d == 0 ? (hi ? nx - 1 : 0) : p, bey = d == 0 ? p : (hi ? ny - 1 : 0);
        const int gex = d == 0 ? (hi ? nx : -1) : p, gey = d == 0 ? p : (hi ? ny : -1);
        const long long eb = storage_elem(nx, ny, bex, bey, ez), eg = storage_elem(nx, ny, gex, gey, ez);
        for (int t2 = 0; t2 < Nq; ++t2)
          for (int t1 = 0; t1 < Nq; ++t1) {
            // face nodes: on an x side (i = a; j = t1, k = t2), on a y side (j = a; i = t1, k = t2); the
            // ghost on side s holds the neighbour's face on side s ^ 1, which is node index N - a here
            const int ns = d == 0 ? a + Nq * (t1 + Nq * t2) : t1 + Nq * (a + Nq * t2);
            const int ag = N - a;
            const int nr = d == 0 ? ag + Nq * (t1 + Nq * t2) : t1 + Nq * (ag + Nq * t2);
            send[s].push_back(eb * Np + ns);
            recv[s].push_back(eg * Np + nr);
          }
      }
  }
  return true;
}

// ---- kernels of the exchange and of the state's scatter / gather

// One array taking part in an exchange: planes [first, first + n) of an
// array with `planes` planes per element and `stride` entries per plane.
struct HaloField {
  void *base;
  int planes, first, n, stride;
};
struct HaloSet {
  HaloField f[2];
  int nf;     // arrays
  int width;  // values per face node (sum of n)
  int Np;
};

template <typename T>
__global__ void k_halo_pack(const HaloSet H, const long long *__restrict__ idx, long long count, T *__restrict__ buf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const long long g = idx[i];
    const long long e = g / H.Np;
    const int n = (int)(g - e * H.Np);
    int o = 0;
    for (int a = 0; a < H.nf; ++a) {
      const HaloField &F = H.f[a];
      const T *src = static_cast<const T *>(F.base);
      for (int p = 0; p < F.n; ++p) buf[i * H.width + o + p] = src[(e * F.planes + F.first + p) * F.stride + n];
      o += F.n;
    }
  }
}

template <typename T>
__global__ void k_halo_unpack(const HaloSet H, const long long *__restrict__ idx, long long count,
                              const T *__restrict__ buf) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
    const long long g = idx[i];
    const long long e = g / H.Np;
    const int n = (int)(g - e * H.Np);
    int o = 0;
    for (int a = 0; a < H.nf; ++a) {
      const HaloField &F = H.f[a];
      T *dst = static_cast<T *>(F.base);
      for (int p = 0; p < F.n; ++p) dst[(e * F.planes + F.first + p) * F.stride + n] = buf[i * H.width + o + p];
      o += F.n;
    }
  }
}

// Whole-mesh state [E][6][Np] <-> a partition's interior (storage layout):
// dir 0 scatters global into the partition, dir 1 gathers.
__global__ void k_part_copy(double *__restrict__ glob, double *__restrict__ loc, int gnex, int gney, int gx0, int gy0,
                            int nx, int ny, int nez, int Np, int dir) {
  const long long total = (long long)nx * ny * nez * Np;
  for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const long long el = q / Np;
    const int n = (int)(q - el * Np);
    const int ex = (int)(el % nx), ey = (int)((el / nx) % ny), ez = (int)(el / ((long long)nx * ny));
    const long long es = (ex + 1) + (long long)(nx + 2) * ((ey + 1) + (long long)(ny + 2) * ez);
    const long long eg = (gx0 + ex) + (long long)gnex * ((gy0 + ey) + (long long)gney * ez);
    for (int v = 0; v < 6; ++v) {
      double *g = glob + (eg * 6 + v) * Np + n;
      double *l = loc + (es * 6 + v) * Np + n;
      if (dir == 0)
        *l = *g;
      else
        *g = *l;
    }
  }
}

int blocks_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 148 * 8) b = 148 * 8;
  return (int)(b < 1 ? 1 : b);
}

// The arrays of exchange A (state and thermodynamic fields, from buffer set
// `which`: FP64 Q[which] / TH64[which], FP32 S32[which] / TH32[which]) or B
// (F2, direction d) of partition h.
HaloSet halo_set(cmles_handle h, int which, bool B, int d) {
  HaloSet H;
  memset(&H, 0, sizeof(H));
  H.Np = h->Np;
  const int stride = h->fp32 ? np32(h->N) : h->Np;
  if (!B) {
    H.nf = 2;
    H.f[0] = {h->fp32 ? (void *)h->S32[which] : (void *)h->Q[which], 6, 0, 6, stride};
    H.f[1] = {h->fp32 ? (void *)h->TH32[which] : (void *)h->TH64[which], 4, 0, 4, stride};
    H.width = 10;
  } else {
    H.nf = 1;
    H.f[0] = {h->fp32 ? (void *)h->F2_32 : (void *)h->F2, 15, 5 * d, 5, stride};
    H.width = 5;
  }
  return H;
}

// One halo exchange: pack every partition's sides, copy each into the
// receiving partition's buffer, unpack.  which[p]: the buffer set of exchange
// A per partition (ignored for B).
cmles_status exchange(cmles_group g, bool B, const std::vector<int> &which) {
  const int P = (int)g->part.size();
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    for (int s = 0; s < 4; ++s) {
      auto &sd = g->side[p * 4 + s];
      if (sd.nb < 0) continue;
      const HaloSet H = halo_set(h, which[p], B, s >> 1);
      LaunchScope ls(h, 2, 1);
      if (h->fp32)
        k_halo_pack<float><<<blocks_for(sd.count, 256), 256, 0, g->stream>>>(H, sd.send_idx, sd.count,
                                                                             (float *)sd.send_buf);
      else
        k_halo_pack<double><<<blocks_for(sd.count, 256), 256, 0, g->stream>>>(H, sd.send_idx, sd.count,
                                                                              (double *)sd.send_buf);
      GCK(cudaGetLastError());
    }
  }
  for (int p = 0; p < P; ++p)
    for (int s = 0; s < 4; ++s) {
      auto &sd = g->side[p * 4 + s];
      if (sd.nb < 0) continue;
      auto &rd = g->side[sd.nb * 4 + (s ^ 1)];
      const size_t bytes = (size_t)sd.count * (B ? 5 : 10) * (g->part[p]->fp32 ? 4 : 8);
      GCK(cudaMemcpyAsync(rd.recv_buf, sd.send_buf, bytes, cudaMemcpyDeviceToDevice, g->stream));
    }
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    for (int s = 0; s < 4; ++s) {
      auto &sd = g->side[p * 4 + s];
      if (sd.nb < 0) continue;
      const HaloSet H = halo_set(h, which[p], B, s >> 1);
      LaunchScope ls(h, 2, 1);
      if (h->fp32)
        k_halo_unpack<float><<<blocks_for(sd.count, 256), 256, 0, g->stream>>>(H, sd.recv_idx, sd.count,
                                                                               (const float *)sd.recv_buf);
      else
        k_halo_unpack<double><<<blocks_for(sd.count, 256), 256, 0, g->stream>>>(H, sd.recv_idx, sd.count,
                                                                                (const double *)sd.recv_buf);
      GCK(cudaGetLastError());
    }
  }
  return CMLES_OK;
}

cmles_status part_copy(cmles_group g, int p, const double *glob, double *loc, int dir) {
  cmles_handle h = g->part[p];
  const cmles_host::PartSpec &ps = g->spec[p];
  const long long n = h->nodes;
  LaunchScope ls(h, 2, 1);
  k_part_copy<<<blocks_for(n, 256), 256, 0, g->stream>>>(const_cast<double *>(glob), loc, g->mesh.nex, g->mesh.ney,
                                                         ps.gx0, ps.gy0, h->mesh.nex, h->mesh.ney, h->mesh.nez,
                                                         h->Np, dir);
  GCK(cudaGetLastError());
  return CMLES_OK;
}

// a partition handle's status as the group's
cmles_status pcheck(cmles_group g, int p, cmles_status st) {
  if (st != CMLES_OK) g->err = "partition " + std::to_string(p) + ": " + g->part[p]->err;
  return st;
}

// The gradient pass of every partition, exchange B, then the flux pass of
// every partition.  in[p]: the state buffer set; Rout[p]: FP64 tendency
// output (no update) or null; with update the new state goes to 1 - in[p].
cmles_status passes(cmles_group g, const std::vector<int> &in, const std::vector<double *> &Rout, const StageCoef &sc,
                    bool update) {
  const int P = (int)g->part.size();
  {
    cmles_status st = exchange(g, false, in);
    if (st != CMLES_OK) return st;
  }
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    LaunchScope ls(h, 0, 1);
    if (h->fp32)
      GCK(launch_grad32(h->S32[in[p]], h->TH32[in[p]], h->F2_32, h->K, g->stream));
    else
      GCK(launch_grad64(h->Q[in[p]], h->TH64[in[p]], h->F2, h->K, g->stream));
  }
  {
    cmles_status st = exchange(g, true, in);
    if (st != CMLES_OK) return st;
  }
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    const int i = in[p];
    LaunchScope ls(h, 1, 1);
    if (h->fp32)
      GCK(launch_rhs32(h->S32[i], h->F2_32, h->TH32[i], h->dQ32, h->Q[0], update ? h->S32[1 - i] : nullptr,
                       update ? h->TH32[1 - i] : nullptr, Rout[p], sc, update, h->K, g->stream));
    else
      GCK(launch_rhs64(h->Q[i], h->F2, h->TH64[i], update ? h->dQ : Rout[p], update ? h->Q[1 - i] : nullptr,
                       update ? h->TH64[1 - i] : nullptr, sc, update, h->K, g->stream));
  }
  return CMLES_OK;
}

}  // namespace

extern "C" {

cmles_status cmles_halo_plan(const cmles_mesh *mesh, int px, int py, int rank, int neighbour[4], long long count[4],
                             long long *send_index, long long *recv_index) {
  if (!mesh || !neighbour || !count) return CMLES_ERR_ARG;
  if (mesh->N < 1 || mesh->N > 7 || mesh->nex < 1 || mesh->ney < 1 || mesh->nez < 1) return CMLES_ERR_ARG;
  std::vector<long long> send[4], recv[4];
  if (!halo_plan(*mesh, px, py, rank, neighbour, send, recv)) return CMLES_ERR_ARG;
  long long o = 0;
  for (int s = 0; s < 4; ++s) {
    count[s] = (long long)send[s].size();
    for (size_t i = 0; i < send[s].size(); ++i) {
      if (send_index) send_index[o + i] = send[s][i];
      if (recv_index) recv_index[o + i] = recv[s][i];
    }
    o += count[s];
  }
  return CMLES_OK;
}

cmles_status cmles_group_destroy(cmles_group g) {
  if (!g) return CMLES_ERR_ARG;
  for (auto &sd : g->side) {
    void *b[4] = {sd.send_idx, sd.recv_idx, sd.send_buf, sd.recv_buf};
    for (void *x : b)
      if (x) cudaFree(x);
  }
  for (double *b : g->tmpQ)
    if (b) cudaFree(b);
  for (double *b : g->tmpR)
    if (b) cudaFree(b);
  for (cmles_handle h : g->part)
    if (h) cmles_destroy(h);
  delete g;
  return CMLES_OK;
}

cmles_status cmles_group_create(const cmles_mesh *mesh, const cmles_params *params, int px, int py,
                                cmles_group *out) {
  if (!mesh || !params || !out) return CMLES_ERR_ARG;
  *out = nullptr;
  if (px < 1 || py < 1 || px > mesh->nex || py > mesh->ney) return CMLES_ERR_ARG;
  // flat meshes with the explicit integrators, no filter (these are the
  // parts of the path that the partitions run)
  if (mesh->warp || params->integrator == CMLES_ARK2_HEVI || params->filter_order > 0) return CMLES_ERR_ARG;
  cmles_group g = new cmles_group_t();
  g->mesh = *mesh;
  g->prm = *params;
  g->px = px;
  g->py = py;
  const int P = px * py;
  const double hx = mesh->Lx / mesh->nex, hy = mesh->Ly / mesh->ney;
  g->part.assign(P, nullptr);
  g->spec.resize(P);
  g->side.resize((size_t)P * 4);
  g->tmpQ.assign(P, nullptr);
  g->tmpR.assign(P, nullptr);
  for (int p = 0; p < P; ++p) {
    cmles_host::PartSpec &ps = g->spec[p];
    ps.global = *mesh;
    int x0, nx, y0, ny;
    split(mesh->nex, px, p % px, &x0, &nx);
    split(mesh->ney, py, p / px, &y0, &ny);
    ps.gx0 = x0;
    ps.gy0 = y0;
    int nb[4];
    std::vector<long long> send[4], recv[4];
    halo_plan(*mesh, px, py, p, nb, send, recv);
    for (int s = 0; s < 4; ++s) ps.wall[s] = nb[s] < 0 ? 1 : 0;
    cmles_mesh lm = *mesh;
    lm.nex = nx;
    lm.ney = ny;
    lm.x0 = mesh->x0 + x0 * hx;
    lm.y0 = mesh->y0 + y0 * hy;
    lm.Lx = nx * hx;
    lm.Ly = ny * hy;
    cmles_status st = create_handle(&lm, params, &ps, &g->part[p]);
    if (st != CMLES_OK) {
      cmles_group_destroy(g);
      return st;
    }
    cmles_handle h = g->part[p];
    const size_t vbytes = h->fp32 ? 4 : 8;
    for (int s = 0; s < 4; ++s) {
      auto &sd = g->side[p * 4 + s];
      sd.nb = nb[s];
      sd.count = (long long)send[s].size();
      if (sd.nb < 0) continue;
      const size_t ib = sd.count * sizeof(long long), bb = (size_t)sd.count * 10 * vbytes;
      if (dalloc(h, (void **)&sd.send_idx, ib) != CMLES_OK || dalloc(h, (void **)&sd.recv_idx, ib) != CMLES_OK ||
          dalloc(h, &sd.send_buf, bb) != CMLES_OK || dalloc(h, &sd.recv_buf, bb) != CMLES_OK ||
          cudaMemcpy(sd.send_idx, send[s].data(), ib, cudaMemcpyHostToDevice) != cudaSuccess ||
          cudaMemcpy(sd.recv_idx, recv[s].data(), ib, cudaMemcpyHostToDevice) != cudaSuccess) {
        cmles_group_destroy(g);
        return CMLES_ERR_OOM;
      }
      g->halo_bytes_stage += (long long)sd.count * 15 * vbytes;
    }
    if (h->fp32) {
      if (dalloc(h, (void **)&g->tmpQ[p], (size_t)h->snodes * 6 * sizeof(double)) != CMLES_OK ||
          dalloc(h, (void **)&g->tmpR[p], (size_t)h->snodes * 6 * sizeof(double)) != CMLES_OK) {
        cmles_group_destroy(g);
        return CMLES_ERR_OOM;
      }
    }
  }
  *out = g;
  return CMLES_OK;
}

const char *cmles_group_last_error_message(cmles_group g) { return g ? g->err.c_str() : "null group"; }

cmles_status cmles_group_set_stream(cmles_group g, void *stream) {
  if (!g) return CMLES_ERR_ARG;
  g->stream = (cudaStream_t)stream;
  for (cmles_handle h : g->part) cmles_set_stream(h, stream);
  return CMLES_OK;
}

cmles_status cmles_group_set_reference(cmles_group g, const double *rho_r_host, const double *p_r_host,
                                       const double *qt_r_host, size_t n) {
  if (!g) return CMLES_ERR_ARG;
  for (int p = 0; p < (int)g->part.size(); ++p) {
    cmles_status st = pcheck(g, p, cmles_set_reference(g->part[p], rho_r_host, p_r_host, qt_r_host, n));
    if (st != CMLES_OK) return st;
  }
  return CMLES_OK;
}

cmles_status cmles_group_set_closure_weights(cmles_group g, const float *params_host, size_t n) {
  if (!g) return CMLES_ERR_ARG;
  for (int p = 0; p < (int)g->part.size(); ++p) {
    cmles_status st = pcheck(g, p, cmles_set_closure_weights(g->part[p], params_host, n));
    if (st != CMLES_OK) return st;
  }
  return CMLES_OK;
}

cmles_status cmles_group_set_state(cmles_group g, const double *Q_dev) {
  if (!g || !Q_dev) return gfail(g, CMLES_ERR_ARG, "cmles_group_set_state: null argument");
  for (int p = 0; p < (int)g->part.size(); ++p) {
    cmles_handle h = g->part[p];
    cmles_status st = part_copy(g, p, Q_dev, h->Q[h->cur], 0);
    if (st != CMLES_OK) return st;
    h->shadow_valid = false;
  }
  return CMLES_OK;
}

cmles_status cmles_group_get_state(cmles_group g, double *Q_dev) {
  if (!g || !Q_dev) return gfail(g, CMLES_ERR_ARG, "cmles_group_get_state: null argument");
  for (int p = 0; p < (int)g->part.size(); ++p) {
    cmles_handle h = g->part[p];
    cmles_status st = part_copy(g, p, Q_dev, h->Q[h->cur], 1);
    if (st != CMLES_OK) return st;
  }
  return CMLES_OK;
}

cmles_status cmles_group_tendency(cmles_group g, const double *Q_dev, double *RHS_dev) {
  if (!g || !Q_dev || !RHS_dev) return gfail(g, CMLES_ERR_ARG, "cmles_group_tendency: null argument");
  const int P = (int)g->part.size();
  std::vector<int> in(P);
  std::vector<double *> R(P);
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    if (!h->have_ref) return gfail(g, CMLES_ERR_STATE, "cmles_group_tendency: reference state not set");
    if (h->prm.closure == CMLES_CLOSURE_MLP && !h->have_mlp)
      return gfail(g, CMLES_ERR_STATE, "cmles_group_tendency: closure weights not set");
    // the input state into idle buffers; the partitions' own states are untouched
    cmles_status st;
    if (h->fp32) {
      if ((st = part_copy(g, p, Q_dev, g->tmpQ[p], 0)) != CMLES_OK) return st;
      in[p] = 1 - h->scur;
      if ((st = pcheck(g, p, write_shadow(h, g->tmpQ[p], in[p]))) != CMLES_OK) return st;
      R[p] = g->tmpR[p];
    } else {
      in[p] = 1 - h->cur;
      if ((st = part_copy(g, p, Q_dev, h->Q[in[p]], 0)) != CMLES_OK) return st;
      if ((st = pcheck(g, p, write_thermo64(h, h->Q[in[p]], h->TH64[in[p]]))) != CMLES_OK) return st;
      R[p] = h->dQ;  // the step's register: every step's first stage starts it afresh
    }
  }
  const StageCoef sc = {0.0, 0.0, 0.0, 0, 0.f, 0.f, 0.f, 1};
  cmles_status st = passes(g, in, R, sc, false);
  if (st != CMLES_OK) return st;
  for (int p = 0; p < P; ++p)
    if ((st = part_copy(g, p, RHS_dev, R[p], 1)) != CMLES_OK) return st;
  return CMLES_OK;
}

cmles_status cmles_group_step(cmles_group g, int nsteps) {
  if (!g || nsteps < 0) return gfail(g, CMLES_ERR_ARG, "cmles_group_step: bad argument");
  const int P = (int)g->part.size();
  for (int p = 0; p < P; ++p) {
    cmles_handle h = g->part[p];
    if (!h->have_ref) return gfail(g, CMLES_ERR_STATE, "cmles_group_step: reference state not set");
    if (h->prm.closure == CMLES_CLOSURE_MLP && !h->have_mlp)
      return gfail(g, CMLES_ERR_STATE, "cmles_group_step: closure weights not set");
    cmles_status st = pcheck(g, p, ensure_shadow(h));
    if (st != CMLES_OK) return st;
  }
  const double *TA, *TB;
  const int nst = lsrk_tables(g->part[0], &TA, &TB);
  const double dt = g->prm.dt;
  std::vector<int> in(P);
  std::vector<double *> R(P, nullptr);
  for (int s = 0; s < nsteps; ++s) {
    for (int k = 0; k < nst; ++k) {
      StageCoef sc = {TA[k], TB[k], dt, k == nst - 1, (float)TA[k], (float)TB[k], (float)dt, TA[k] == 0.0};
      for (int p = 0; p < P; ++p) in[p] = g->part[p]->fp32 ? g->part[p]->scur : g->part[p]->cur;
      cmles_status st = passes(g, in, R, sc, true);
      if (st != CMLES_OK) return st;
      for (int p = 0; p < P; ++p) {
        cmles_handle h = g->part[p];
        if (h->fp32)
          h->scur = 1 - h->scur;
        else
          h->cur = 1 - h->cur;
      }
    }
    for (int p = 0; p < P; ++p) {
      g->part[p]->steps += 1;
      g->part[p]->time += dt;
    }
  }
  return CMLES_OK;
}

cmles_status cmles_group_diagnostics(cmles_group g, cmles_diag *out) {
  if (!g || !out) return gfail(g, CMLES_ERR_ARG, "cmles_group_diagnostics: null argument");
  memset(out, 0, sizeof(*out));
  double nonfinite = 0.0;
  for (int p = 0; p < (int)g->part.size(); ++p) {
    cmles_handle h = g->part[p];
    const double J = h->K.hx * h->K.hy * h->K.hz / 8.0;
    {
      LaunchScope ls(h, 2, 2);
      GCK(launch_budgets(h->Q[h->cur], h->E, h->Np, h->wq, J, h->partials, h->budget_nblocks, h->budget_out,
                         g->stream, nullptr, h->mesh.nex, h->mesh.ney));
    }
    double res[7];
    int flags[16];
    GCK(cudaMemcpyAsync(res, h->budget_out, 7 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    GCK(cudaMemcpyAsync(flags, h->flags, 16 * sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    GCK(cudaMemsetAsync(h->flags, 0, 16 * sizeof(int), g->stream));
    GCK(cudaStreamSynchronize(g->stream));
    // the allreduce of a multi-GPU run: sums over the partitions
    for (int v = 0; v < 6; ++v) out->budget[v] += res[v];
    nonfinite += res[6];
    out->satadj_failures += flags[0];
    out->tc_timeouts += flags[1];
    out->cold_saturated += flags[2];
    out->time = h->time;
    out->steps = h->steps;
  }
  out->nonfinite = nonfinite > 0.0 ? 1 : 0;
  if (out->nonfinite) return gfail(g, CMLES_ERR_NONFINITE, "state holds non-finite values");
  if (out->satadj_failures) return gfail(g, CMLES_ERR_SATADJ, "saturation adjustment did not converge");
  if (out->tc_timeouts) return gfail(g, CMLES_ERR_TIMEOUT, "a tensor-core completion wait gave up");
  return CMLES_OK;
}

long long cmles_group_halo_bytes(cmles_group g) { return g ? g->halo_bytes_stage : -1; }

}  // extern "C"
