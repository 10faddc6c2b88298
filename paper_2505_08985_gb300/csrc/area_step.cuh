// Projected-area requests inside a serving step (serve.cu builds the table,
// projarea.cu runs it): each request of the step is one descriptor, and the
// step's kernels read the request count from the device table, so one
// captured graph serves any mix.
#pragma once

#include "common.cuh"

namespace pndf {

// One projected-area request of a step: its record (x, S), its unit
// direction (3 floats), where its P goes, and its map's index.
struct AreaReq {
    const pndf_query *q;
    const float *w;
    float *out;
    int32_t map;
    int32_t pad;
};

// Bands of kBand quad rows per request bound a step's partial sums.
int area_max_bands(int n);

// The step's projected-area kernels: band counts, their scan, the band
// integrals and the fixed-order per-request sums, for the *count (<= cap,
// read on the device) descriptors at areq; off has cap + 1 words, part
// cap * max_bands float2, cursor one word.
cudaError_t launch_area_step(int texel_fmt, const MapDesc *maps, int nmaps, const uint32_t *count,
                             const AreaReq *areq, int cap, uint32_t *off, float2 *part, unsigned int *cursor,
                             cudaStream_t s);

}  // namespace pndf
