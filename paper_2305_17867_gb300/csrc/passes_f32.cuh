// Warp-per-box kernels of the upward and downward passes of 3D uniform trees
// (passes_f32.cu): P2M and L2P in float, M2M and L2L in float, double-word float or FP64.  Each launcher returns false,
// launching nothing, when the plan is outside what they cover (d != 3, an
// order other than 4, 6, 8, 10, 12, 16, or no box-relative point copy).
#pragma once

#include "fmm_internal.cuh"

bool passes_f32_order(int p);
bool launch_p2m_f32(const fmm_plan_s* P, const Workspace& ws, cudaStream_t st);
// the same for the leaves (level >= 2) of an adaptive tree, from its FP64 points
struct ATree;
bool launch_ap2m_f32(const fmm_plan_s* P, const Workspace& ws, const ATree& t, cudaStream_t st);
// M2M from level l + 1 into level l, L2L from level l into level l + 1, in
// float, double-word float (dwf.cuh) or FP64 arithmetic
enum ShiftArith { kShiftF32, kShiftDW, kShiftF64 };
bool launch_m2m_warp(const fmm_plan_s* P, const Workspace& ws, int l, ShiftArith a,
                     cudaStream_t st);
bool launch_l2l_warp(const fmm_plan_s* P, const Workspace& ws, int l, ShiftArith a,
                     cudaStream_t st);
// far field at the targets of the leaves, added to phi (and grad)
bool launch_l2p_f32(const fmm_plan_s* P, const Workspace& ws, double* phi, double* grad,
                    cudaStream_t st);
