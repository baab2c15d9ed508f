// The fp32 pair passes and gathers of force.cu, compiled as a translation unit of its own
// (a unit of its own name, so that the kernels of force.cu's internal namespace get names of
// their own in each object).
#define MD_FORCE_PART 2
#include "force.cu"
