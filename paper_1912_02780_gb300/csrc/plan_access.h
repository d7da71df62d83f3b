// Internal accessors of a plan's device state for library components built
// on top of the plan (the L-BFGS isometry optimiser); not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include "../../include/hotrg.h"

namespace hotrg {

cudaStream_t plan_stream(hotrg_plan p);
int plan_sms(hotrg_plan p);
int* plan_err(hotrg_plan p);                    // device error word (two ints)
double* plan_isometry(hotrg_plan p, int k);     // w_k: X'_k rows of X_k^2 (row a = vector a)
const double* plan_wbar(hotrg_plan p, int k);   // d(ln Z/N)/d w_k of the last backward, same layout
const double* plan_T0(hotrg_plan p);            // the site tensor of the last forward
const double* plan_lnz(hotrg_plan p);           // device ln Z/N of the last forward
bool plan_has_forward(hotrg_plan p);
bool plan_w_given(hotrg_plan p);
int plan_given_steps(hotrg_plan p);
int plan_steps_run(hotrg_plan p);
hotrg_status plan_fail(hotrg_plan p, hotrg_status s, const char* msg);

}  // namespace hotrg
