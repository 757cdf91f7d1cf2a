// Host-side subdomain partition and FETI-DP index maps (built once per mesh, uploaded once).
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace schur {

struct HostMaps {
  Geom g;
  std::vector<int> slot_node;    // [nD] local node of interface slot j
  std::vector<int> node_slot;    // [nl] slot of a local node or -1
  std::vector<int> corner_node;  // [nc] local node of corner c (bit a <=> l_a = s_a)
  std::vector<int> sd_code;      // [nsd] boundary-type code (see local_dirichlet)
  std::vector<int> sd_cls;       // [nsd] class of stored local operators
  std::vector<int> cls_code;     // [ncls] boundary-type code of each class
  std::vector<int> sd_lam;       // [nsd][nD][maxdeg] +-(lambda+1), 0 = none
  std::vector<double> sd_minv;   // [nsd][nD] 1/multiplicity, 0 for Dirichlet slots
  std::vector<int> lam_side;     // [nlam][2] plus side, minus side as (subdomain*nD + slot)
  std::vector<int> sd_corner;    // [nsd][nc] coarse unknown or -1 (Dirichlet)
  // coarse couplings: sd_coarse always (the corners alone without the augmentation); the rest
  // only with the augmented coarse problem
  std::vector<int> sd_coarse;    // [nsd][nq] coarse unknown of each coupling slot (corners, faces) or -1
  std::vector<int> face_sd;      // [nface][2] the lower and the higher subdomain of each face
  std::vector<int> lam_face;     // [nlam] face of the multiplier's subdomain pair, -1 for other pairs
  std::vector<int> face_lam_ptr; // [nface + 1] CSR offsets of the multipliers of each face
  std::vector<int> face_lam;     // multipliers of each face, in increasing order
  std::vector<int> slot_faces;   // [nD] bit f set: slot lies on local face f = 2a + side
  std::vector<int> grp_sd;       // [nsd] subdomains ordered by class
  std::vector<int> grp_ptr;      // [ngrp + 1] groups of at most kApplyGroup subdomains of one class
  int ncls = 0;
};

// Fills maps for the mesh; returns "" on success or a message describing the invalid input.
// augment: also number the faces between subdomains as coarse unknowns (augmented coarse problem).
std::string build_maps(int dim, const int* nel, const int* nsub, int local_mode, HostMaps* m, int augment = 0);

}  // namespace schur
