// adjacency.cuh -- neighbourhood update of the merge (adjacency.cu) and the
// check that a triangulation is the Delaunay triangulation of its points.
#pragma once
#include "ctx.cuh"

namespace gdt {

// Neighbour array of the canonical rows: nbr[r][j] = the row sharing every
// vertex of row r except its j-th, or -1 on the convex hull.
int neighbor_update(dt_ctx* c, int dim, const int32_t* rows, int64_t m, const LinkSources& src, int32_t** nbr);

// The same array from the rows alone (every facet through the facet hash).
// *non_manifold receives the number of facets found in more than two rows.
int match_all_facets(dt_ctx* c, int dim, const int32_t* rows, int64_t m, int32_t** nbr, int64_t* non_manifold);

// Local checks that certify rows (sorted tuples, indices checked) as the
// perturbed Delaunay triangulation of P (input order, n points).
int validate_rows(dt_ctx* c, int dim, const void* P, int64_t n, const int32_t* rows, int64_t m,
                  const int32_t* nbr, int64_t non_manifold, dt_validation* out);

// Rows from a caller: sort each tuple and count out-of-range or repeated indices.
int prepare_rows(dt_ctx* c, int dim, const int32_t* in, int64_t m, int64_t n, int32_t* out, int64_t* bad);

}  // namespace gdt
