// Oracle internals. TEST INFRASTRUCTURE ONLY: nothing in the product path may
// include, link or call this code. It is a plain, slow, obviously-correct CPU
// restatement of the cellGPU method (Sussman, arXiv 1702.02939) used to check
// the CUDA path. It shares no code with the CUDA library.
#pragma once
#include <cstdint>
#include <vector>

namespace cgo {

typedef __int128 i128;
typedef unsigned __int128 u128;

// A point of the (tiled) Delaunay input in integer grid units.
// x_real = X * 2^-q exactly (positions live on a dyadic grid, see snap).
struct Pt {
  int64_t X, Y;
  int32_t tag;  // cell index (user order); -1 for a super-triangle vertex
  int32_t ox, oy;  // periodic image offset of this copy
  int64_t key;  // symbolic-perturbation priority (larger = dominant)
};

// exact.cpp ----------------------------------------------------------------
int orient2d_exact(const Pt& a, const Pt& b, const Pt& c);
int incircle_exact(const Pt& a, const Pt& b, const Pt& c, const Pt& d);
int incircle_sos(const Pt& a, const Pt& b, const Pt& c, const Pt& d);

// delaunay.cpp -------------------------------------------------------------
struct Ring {
  // CCW neighbours of a cell: tag and periodic offset relative to the cell.
  std::vector<int32_t> tag;
  std::vector<int32_t> ox, oy;
};
// Delaunay triangulation of `pts` (Bowyer-Watson, exact predicates).
// Fills rings for every point whose `central` flag is set.  Returns 0 or a
// negative error code.  With allow_open, points on the hull of a plain point
// set (open fans) get an empty ring instead of an error.
int bowyer_watson_rings(const std::vector<Pt>& pts, const std::vector<char>& central,
                        std::vector<Ring>& rings_out, bool allow_open = false);

// philox.cpp ----------------------------------------------------------------
void philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

}  // namespace cgo
