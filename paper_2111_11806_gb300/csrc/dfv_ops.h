// dfv_ops.h -- host-side table of launchers for one (precision, dimension,
// materials, solid) combination.  The C ABI in dfv_api.cu picks a table at
// grid creation and issues every launch of a step through it.
#pragma once

#include <cuda_runtime.h>

#include "dfv_device.cuh"

namespace dfv {

struct StageArgs;

struct Ops {
    int nvar;
    int threads_stage;
    int elem_bytes;
    cudaError_t (*prepare)();
    dim3 (*stage_grid)(const GridP &);
    // fin_mode != 0 (stepped probe only): the same launch runs the deferred
    // finalize of the previous step with that mode
    cudaError_t (*seed)(const GridP &, void *U, void *scratch, Ctl *ctl, int fin_mode, cudaStream_t);
    // next: the seeding before this stage 1 took its box from ctl->rnext
    cudaError_t (*stage)(int stage, const GridP &, const void *in, const void *un, void *out, Ctl *ctl,
                         double *partials, int want_force, int next, cudaStream_t);
    cudaError_t (*cfl)(const GridP &, const void *U, double *partials, int nblocks, cudaStream_t);
    cudaError_t (*prim_to_cons)(const GridP &, const double *prim, long long ppitch, void *U, cudaStream_t);
    cudaError_t (*cons_to_prim)(const GridP &, const void *U, double *prim, long long ppitch, cudaStream_t);
    cudaError_t (*cons_to_f64)(const GridP &, const void *U, double *out, long long ppitch, int nvar, cudaStream_t);
};

// nullptr when the combination is not built.  One translation unit per
// (precision, dimension, materials) so that the build compiles them in
// parallel (dfv_inst_tu.cu, compiled once per combination).
const Ops *ops_f32_d1_n1(int solid);
const Ops *ops_f32_d1_n2(int solid);
const Ops *ops_f32_d1_n3(int solid);
const Ops *ops_f32_d2_n1(int solid);
const Ops *ops_f32_d2_n2(int solid);
const Ops *ops_f32_d2_n3(int solid);
const Ops *ops_f32_d3_n1(int solid);
const Ops *ops_f32_d3_n2(int solid);
const Ops *ops_f32_d3_n3(int solid);
const Ops *ops_f64_d1_n1(int solid);
const Ops *ops_f64_d1_n2(int solid);
const Ops *ops_f64_d1_n3(int solid);
const Ops *ops_f64_d2_n1(int solid);
const Ops *ops_f64_d2_n2(int solid);
const Ops *ops_f64_d2_n3(int solid);
const Ops *ops_f64_d3_n1(int solid);
const Ops *ops_f64_d3_n2(int solid);
const Ops *ops_f64_d3_n3(int solid);

inline const Ops *ops_for(int precision_fp32, int dim, int nmat, int solid)
{
    typedef const Ops *(*Fn)(int);
    static const Fn f32[3][3] = {{ops_f32_d1_n1, ops_f32_d1_n2, ops_f32_d1_n3},
                                 {ops_f32_d2_n1, ops_f32_d2_n2, ops_f32_d2_n3},
                                 {ops_f32_d3_n1, ops_f32_d3_n2, ops_f32_d3_n3}};
    static const Fn f64[3][3] = {{ops_f64_d1_n1, ops_f64_d1_n2, ops_f64_d1_n3},
                                 {ops_f64_d2_n1, ops_f64_d2_n2, ops_f64_d2_n3},
                                 {ops_f64_d3_n1, ops_f64_d3_n2, ops_f64_d3_n3}};
    if (dim < 1 || dim > 3 || nmat < 1 || nmat > 3) return nullptr;
    return (precision_fp32 ? f32 : f64)[dim - 1][nmat - 1](solid);
}

// Grid-stride launches use at most this many blocks of 256 threads.
inline int gs_blocks(long long n)
{
    long long b = (n + 255) / 256;
    const long long cap = 152LL * 16;
    return (int)(b < 1 ? 1 : (b > cap ? cap : b));
}

}  // namespace dfv
