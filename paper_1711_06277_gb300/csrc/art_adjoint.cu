// art_adjoint.cu -- placeholder replaced by the reverse-sweep kernels.
#include "art.h"
extern "C" int art_trace_backward(art_grid*, const art_params*, const float*, float*, double*,
                                  art_stats*)
{
    return ART_ESTATE;
}
