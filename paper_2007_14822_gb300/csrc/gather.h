// Tile gather (see gather.cu): GEMM operand tiles assembled from weighted
// sums of strided sub-blocks.
#pragma once

#include "tnh_internal.h"

namespace tnh {

constexpr int kGatherRows = 128, kGatherCols = 64;   // one operand tile

struct GatherTerm {
    double coef;
    int64_t off;     // source element of the segment's (0, 0)
    int64_t rs, cs;  // source strides along the segment's rows / columns
    float coef32;    // coef for the float32 arithmetic of the split formats
};
struct GatherSeg {
    int r0, c0, nr, nc;   // rectangle inside the tile
    int t0, t1;           // its terms
};
struct GatherTile {
    int task, mi, ki;     // operand tile (mi, ki) of a GEMM task
    int seg0, seg1;       // its segments
};

// One operand: every tile of every task, in order (a tile with no segment
// is written as zeros).
struct GatherJob {
    std::vector<GatherTile> tiles;
    std::vector<GatherSeg> segs;
    std::vector<GatherTerm> terms;
    int ntiles = 0;
    DevBuf d_tiles, d_segs, d_terms;
    void upload_all(cudaStream_t s);
};

// Fused two-site MPO step (S2+S3). A cell is one pair (a'-sector, b-sector):
// all its inputs (T1 sub-blocks) and outputs (T3 sub-blocks, placed in the
// S4 operand) are Da x Db matrices. Every output is a weighted sum of inputs
// (the nonzero entries of W12). One thread owns four consecutive columns of
// one row of the cell (a "quad"; rows of T1 sub-blocks and columns of T3
// sub-blocks start at multiples of 4) and forms them for every output of
// the cell; one CTA owns kW12Threads quads.
constexpr int kW12Threads = 128;
struct W12Cell { int in0, nin, out0, nout, Da, Db; };
struct W12In { int64_t base; int64_t ld; };
struct W12Out { int task, row0, col0, t0, t1; };
struct W12Term { int64_t base; double coef; float coef32; int ld; };   // input T1 sub-block (base, row pitch)
struct W12Cta { int cell, q0; };
struct W12Job {
    std::vector<W12Cell> cells;
    std::vector<W12In> ins;
    std::vector<W12Out> outs;
    std::vector<W12Term> terms;
    std::vector<W12Cta> ctas;
    DevBuf d_cells, d_ins, d_outs, d_terms, d_ctas;
    void upload_all(cudaStream_t s);
};
// The S4 GEMM with its operand A formed in the kernel from T1 (float32) by
// the gather job (atiles, asegs, aterms) over the operand's tile numbering,
// three-plane split; B packed. Same output conventions as launch_gemm_tc.
void launch_gemm_tc_fused(const GemmTask* d_tasks, int ntasks, int total_tiles, const GatherTile* atiles,
                          const GatherSeg* asegs, const GatherTerm* aterms, const float* asrc, const uint16_t* B,
                          double* C, int num_sms, int* err, cudaStream_t s, const int64_t* row_off);

// src: T1 (float64 or float32); dst: S4 operand A in the format of planes.
void launch_w12(const W12Job& J, const OpGeom* d_geom, const double* src, void* dst, int planes, cudaStream_t s);
void launch_w12(const W12Job& J, const OpGeom* d_geom, const float* src, void* dst, int planes, cudaStream_t s);

// planes 0: float64 rows, OpGeom {element offset, row pitch}; planes 1..3:
// split-bfloat16 tiles, OpGeom {tile offset, tiles along K}.
void launch_gather(const GatherJob& J, const OpGeom* d_geom, const double* src, void* dst, int planes,
                   cudaStream_t s, const char* name);
void launch_gather(const GatherJob& J, const OpGeom* d_geom, const float* src, void* dst, int planes,
                   cudaStream_t s, const char* name);

}  // namespace tnh
