// Subdomain partition and the FETI-DP index maps of Sec. 5 (arXiv 1312.5653):
//  * non-overlapping subdomains (Figure 1), corner nodes primal;
//  * the signed Boolean jump operator B^s of Eq. continuitycondition, one multiplier per pair of
//    subdomains sharing a non-corner interface node (fully redundant where more than two share,
//    i.e. on 3D subdomain edges), +1 on the lower-numbered subdomain, -1 on the other;
//  * W = (sum_s B^s B^s^T)^+ of Eq. WS reduces to scaling each slot by 1/multiplicity.
#include "maps.h"

#include <algorithm>
#include <cstdlib>
#include <map>

namespace schur {

std::string build_maps(int dim, const int* nel, const int* nsub, int local_mode, HostMaps* m, int augment) {
  if (dim != 2 && dim != 3) return "dim must be 2 or 3";
  Geom& g = m->g;
  g = Geom();
  g.dim = dim;
  for (int a = 0; a < 3; ++a) {
    g.nel[a] = a < dim ? nel[a] : 1;
    g.nsub[a] = a < dim ? nsub[a] : 1;
    if (a < dim) {
      if (g.nel[a] < 2 || g.nsub[a] < 1) return "nel must be >= 2 and nsub >= 1 on every axis";
      if (g.nel[a] % g.nsub[a]) return "nel must be a multiple of nsub on every axis";
      g.s[a] = g.nel[a] / g.nsub[a];
      if (g.s[a] < 2) return "subdomains need at least 2 elements per axis";
      g.h[a] = 1.0 / g.nel[a];
    } else {
      g.s[a] = 0;
      g.h[a] = 1.0;
    }
  }
  g.nsd = 1;
  g.nl = 1;
  g.ni = 1;
  g.n = 1;
  g.ncor = 1;
  for (int a = 0; a < dim; ++a) {
    g.nsd *= g.nsub[a];
    g.nl *= g.s[a] + 1;
    g.ni *= g.s[a] - 1;
    g.n *= (long long)(g.nel[a] - 1);
    g.ncg[a] = g.nsub[a] - 1;
    g.ncor *= g.ncg[a];
  }
  if (g.n > (1LL << 31) - 1) return "mesh too large";
  g.lL = g.s[dim - 1] + 1;
  g.lb = g.nl / g.lL;
  g.iL = g.s[dim - 1] - 1;
  g.ib = g.ni / g.iL;
  g.nc = 1 << dim;
  g.maxdeg = dim == 2 ? 1 : 3;
  if (g.ncor > 0) {
    g.cL = g.ncg[dim - 1];
    g.cb = g.ncor / g.cL;
  } else {
    g.cL = 0;
    g.cb = 0;
  }
  int ext[3] = {g.s[0] + 1, g.s[1] + 1, dim == 3 ? g.s[2] + 1 : 1};

  // interface slots and corners (same lists for every subdomain)
  m->slot_node.clear();
  m->node_slot.assign(g.nl, -1);
  m->corner_node.assign(g.nc, -1);
  for (int p = 0; p < g.nl; ++p) {
    int l[3];
    idx2crd(p, ext, dim, l);
    if (local_vertex(l, g.s, dim)) {
      int c = 0;
      for (int a = 0; a < dim; ++a) c |= (l[a] == g.s[a]) << a;
      m->corner_node[c] = p;
    } else if (local_on_boundary(l, g.s, dim)) {
      m->node_slot[p] = (int)m->slot_node.size();
      m->slot_node.push_back(p);
    }
  }
  g.nD = (int)m->slot_node.size();

  // subdomain codes and classes
  m->sd_code.assign(g.nsd, 0);
  m->sd_cls.assign(g.nsd, 0);
  m->cls_code.clear();
  std::map<int, int> code2cls;
  for (int sd = 0; sd < g.nsd; ++sd) {
    int S[3];
    idx2crd(sd, g.nsub, dim, S);
    int code = 0;
    for (int a = 0; a < dim; ++a) {
      if (S[a] == 0) code |= 1 << (2 * a);
      if (S[a] == g.nsub[a] - 1) code |= 1 << (2 * a + 1);
    }
    m->sd_code[sd] = code;
    if (local_mode == 1) {
      auto it = code2cls.find(code);
      if (it == code2cls.end()) {
        int q = (int)m->cls_code.size();
        code2cls[code] = q;
        m->cls_code.push_back(code);
        m->sd_cls[sd] = q;
      } else {
        m->sd_cls[sd] = it->second;
      }
    } else {
      m->sd_cls[sd] = sd;
      m->cls_code.push_back(code);
    }
  }
  m->ncls = (int)m->cls_code.size();
  // groups of subdomains that share their stored operators (class by class, increasing index)
  {
    std::vector<std::vector<int>> by(m->ncls);
    for (int sd = 0; sd < g.nsd; ++sd) by[m->sd_cls[sd]].push_back(sd);
    m->grp_sd.clear();
    m->grp_ptr.assign(1, 0);
    for (const auto& v : by)
      for (size_t i = 0; i < v.size(); i += kApplyGroup) {
        for (size_t k = i; k < v.size() && k < i + kApplyGroup; ++k) m->grp_sd.push_back(v[k]);
        m->grp_ptr.push_back((int)m->grp_sd.size());
      }
  }

  // corners -> coarse unknowns
  m->sd_corner.assign((size_t)g.nsd * g.nc, -1);
  for (int sd = 0; sd < g.nsd; ++sd) {
    int S[3];
    idx2crd(sd, g.nsub, dim, S);
    for (int c = 0; c < g.nc; ++c) {
      int C[3] = {0, 0, 0};
      bool inside = true;
      for (int a = 0; a < dim; ++a) {
        C[a] = S[a] + ((c >> a) & 1) - 1;
        if (C[a] < 0 || C[a] >= g.ncg[a]) inside = false;
      }
      if (inside) m->sd_corner[(size_t)sd * g.nc + c] = crd2idx(C, g.ncg, dim);
    }
  }

  // multipliers: visit subdomains and slots in order; for a slot node shared with subdomains
  // of higher index, create one multiplier per such pair
  m->sd_lam.assign((size_t)g.nsd * g.nD * g.maxdeg, 0);
  m->sd_minv.assign((size_t)g.nsd * g.nD, 0.0);
  m->lam_side.clear();
  {
    // multipliers per subdomain pair and shared node: faces 1, 3D edges 6 per node and 4 owners
    long long est = 0;
    for (int a = 0; a < dim; ++a) {
      long long faces = (long long)(g.nsub[a] - 1);
      for (int b = 0; b < dim; ++b)
        if (b != a) faces *= (long long)(g.nel[b] - 1);
      est += faces;
    }
    m->lam_side.reserve((size_t)(2 * est * (dim == 3 ? 2 : 1) + 16));
  }
  std::vector<int> deg((size_t)g.nsd * g.nD, 0);
  for (int sd = 0; sd < g.nsd; ++sd) {
    int S[3];
    idx2crd(sd, g.nsub, dim, S);
    for (int j = 0; j < g.nD; ++j) {
      int l[3];
      idx2crd(m->slot_node[j], ext, dim, l);
      int G[3] = {0, 0, 0};
      bool dir = false;
      for (int a = 0; a < dim; ++a) {
        G[a] = S[a] * g.s[a] + l[a];
        if (G[a] == 0 || G[a] == g.nel[a]) dir = true;
      }
      if (dir) continue;
      // all subdomains holding global node G, with the node's local coordinates there
      std::pair<int, int> owners[8];  // (subdomain, slot), at most 2^(dim-1) for a non-vertex node
      int nown = 0;
      int cand[3][2], ncand[3];
      for (int a = 0; a < 3; ++a) { ncand[a] = 1; cand[a][0] = 0; }
      for (int a = 0; a < dim; ++a) {
        ncand[a] = 0;
        if (l[a] == 0) {
          cand[a][ncand[a]++] = S[a] - 1;
          cand[a][ncand[a]++] = S[a];
        } else if (l[a] == g.s[a]) {
          cand[a][ncand[a]++] = S[a];
          cand[a][ncand[a]++] = S[a] + 1;
        } else {
          cand[a][ncand[a]++] = S[a];
        }
      }
      for (int i0 = 0; i0 < ncand[0]; ++i0)
        for (int i1 = 0; i1 < ncand[1]; ++i1)
          for (int i2 = 0; i2 < ncand[2]; ++i2) {
            int T[3] = {cand[0][i0], cand[1][i1], dim == 3 ? cand[2][i2] : 0};
            int lt[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) lt[a] = G[a] - T[a] * g.s[a];
            int sdt = crd2idx(T, g.nsub, dim);
            int slot = m->node_slot[crd2idx(lt, ext, dim)];
            if (slot < 0) return "internal error: shared node is not an interface slot";
            if (nown >= 8) return "internal error: too many owners";
            owners[nown++] = {sdt, slot};
          }
      std::sort(owners, owners + nown);
      int mult = nown;
      m->sd_minv[(size_t)sd * g.nD + j] = 1.0 / mult;
      for (int oi = 0; oi < nown; ++oi) {
        const auto& o = owners[oi];
        if (o.first <= sd) continue;
        int lam = (int)(m->lam_side.size() / 2);
        m->lam_side.push_back(sd * g.nD + j);
        m->lam_side.push_back(o.first * g.nD + o.second);
        size_t kp = (size_t)sd * g.nD + j, km = (size_t)o.first * g.nD + o.second;
        if (deg[kp] >= g.maxdeg || deg[km] >= g.maxdeg) return "internal error: slot degree";
        m->sd_lam[kp * g.maxdeg + deg[kp]++] = lam + 1;
        m->sd_lam[km * g.maxdeg + deg[km]++] = -(lam + 1);
      }
    }
  }
  g.nlam = (int)(m->lam_side.size() / 2);

  // coarse couplings: corners, and with the augmentation the faces between subdomains
  g.nq = g.nc;
  g.nco = g.ncor;
  g.nface = 0;
  m->sd_coarse.clear();
  m->face_sd.clear();
  m->lam_face.clear();
  m->face_lam_ptr.clear();
  m->face_lam.clear();
  m->slot_faces.clear();
  if (augment) {
    const int ne = 2 * dim;
    g.nq = g.nc + ne;
    // faces normal to axis a: between S and S + e_a, S_a < nsub[a] - 1; numbered axis by axis,
    // lexicographically over the lower subdomain's coordinates
    int foff[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) {
      foff[a] = g.nface;
      int cnt = g.nsub[a] - 1;
      for (int b = 0; b < dim; ++b)
        if (b != a) cnt *= g.nsub[b];
      g.nface += cnt;
    }
    g.nco = g.ncor + g.nface;
    auto face_of = [&](const int* S, int a) {  // face between S and S + e_a
      int idx = 0, stride = 1;
      for (int b = 0; b < dim; ++b) {
        const int ext = b == a ? g.nsub[b] - 1 : g.nsub[b];
        idx += S[b] * stride;
        stride *= ext;
      }
      return foff[a] + idx;
    };
    m->face_sd.assign((size_t)2 * g.nface, -1);
    m->sd_coarse.assign((size_t)g.nsd * g.nq, -1);
    for (int sd = 0; sd < g.nsd; ++sd) {
      int S[3];
      idx2crd(sd, g.nsub, dim, S);
      for (int c = 0; c < g.nc; ++c) m->sd_coarse[(size_t)sd * g.nq + c] = m->sd_corner[(size_t)sd * g.nc + c];
      for (int a = 0; a < dim; ++a)
        for (int side = 0; side < 2; ++side) {
          int T[3] = {S[0], S[1], S[2]};
          if (side == 0) {
            if (S[a] == 0) continue;
            T[a] = S[a] - 1;  // the face lies between T = S - e_a and S
          } else if (S[a] == g.nsub[a] - 1) {
            continue;
          }
          const int f = face_of(T, a);
          m->sd_coarse[(size_t)sd * g.nq + g.nc + 2 * a + side] = g.ncor + f;
          m->face_sd[2 * f + side] = sd;  // side 1: S is the lower subdomain
        }
    }
    // the face slots of every subdomain's local grid
    m->slot_faces.assign(g.nD, 0);
    for (int j = 0; j < g.nD; ++j) {
      int l[3];
      idx2crd(m->slot_node[j], ext, dim, l);
      int bits = 0;
      for (int a = 0; a < dim; ++a) {
        if (l[a] == 0) bits |= 1 << (2 * a);
        if (l[a] == g.s[a]) bits |= 1 << (2 * a + 1);
      }
      m->slot_faces[j] = bits;
    }
    // multipliers between face neighbours belong to that face's average constraint
    m->lam_face.assign(g.nlam, -1);
    for (int li = 0; li < g.nlam; ++li) {
      const int sp = m->lam_side[2 * li] / g.nD, sm = m->lam_side[2 * li + 1] / g.nD;
      int A[3], B[3];
      idx2crd(sp, g.nsub, dim, A);
      idx2crd(sm, g.nsub, dim, B);
      int axis = -1, dist = 0;
      for (int a = 0; a < dim; ++a) {
        dist += std::abs(A[a] - B[a]);
        if (A[a] != B[a]) axis = a;
      }
      if (dist == 1) m->lam_face[li] = face_of(A, axis);  // the plus side is the lower subdomain
    }
    m->face_lam_ptr.assign(g.nface + 1, 0);
    for (int li = 0; li < g.nlam; ++li)
      if (m->lam_face[li] >= 0) ++m->face_lam_ptr[m->lam_face[li] + 1];
    for (int f = 0; f < g.nface; ++f) m->face_lam_ptr[f + 1] += m->face_lam_ptr[f];
    m->face_lam.assign(m->face_lam_ptr[g.nface], 0);
    std::vector<int> fill(m->face_lam_ptr.begin(), m->face_lam_ptr.end() - 1);
    for (int li = 0; li < g.nlam; ++li)
      if (m->lam_face[li] >= 0) m->face_lam[fill[m->lam_face[li]]++] = li;
  } else {
    m->sd_coarse = m->sd_corner;
  }
  return "";
}

}  // namespace schur

// ------------------------------------------------------------------ host-only C entry points
#include <cstring>

#include "../../include/schur.h"

extern "C" {

int schur_partition(const schur_mesh* mesh, const int* nsub, int local_mode, schur_info_t* info) {
  if (!mesh || !nsub || !info) return SCHUR_EINVAL;
  schur::HostMaps hm;
  if (!schur::build_maps(mesh->dim, mesh->nel, nsub, local_mode, &hm).empty()) return SCHUR_EINVAL;
  std::memset(info, 0, sizeof(*info));
  info->n = hm.g.n;
  info->n_sub = hm.g.nsd;
  info->n_classes = hm.ncls;
  info->n_lambda = hm.g.nlam;
  info->n_coarse = hm.g.ncor;
  info->n_delta = hm.g.nD;
  info->n_local = hm.g.nl;
  return SCHUR_OK;
}

int schur_partition_export(const schur_mesh* mesh, const int* nsub, int local_mode, int which, int* out,
                           long long cap) {
  if (!mesh || !nsub || !out) return SCHUR_EINVAL;
  schur::HostMaps hm;
  if (!schur::build_maps(mesh->dim, mesh->nel, nsub, local_mode, &hm).empty()) return SCHUR_EINVAL;
  const std::vector<int>* v = nullptr;
  if (which == 0) v = &hm.lam_side;
  else if (which == 1) v = &hm.slot_node;
  else if (which == 2) v = &hm.sd_corner;
  else if (which == 3) v = &hm.sd_cls;
  else return SCHUR_EINVAL;
  if ((long long)v->size() > cap) return SCHUR_EINVAL;
  if (!v->empty()) std::memcpy(out, v->data(), v->size() * sizeof(int));
  return SCHUR_OK;
}

}  // extern "C"
