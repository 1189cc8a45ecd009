// qt_pass_grp.cu -- the register-resident fused pass with merged phase groups.
//
// The kernels of qt_pass_reg.cu instantiated with support for RC_PH_GROUP
// ops (runs of phases merged by the layout planner), in a translation unit
// of their own so that both sets compile in parallel and passes without
// groups keep running code that has none.  Entry point:
// launch_pass_reg_groups, called by launch_pass_reg for passes with
// DevPass::groups set.
#define QT_PASS_PHASE_GROUPS 1
#include "qt_pass_reg.cu"
