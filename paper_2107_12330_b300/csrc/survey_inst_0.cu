// survey_inst_0.cu -- instantiations of the survey launch for feature sets 0..7
// (survey_kernels.cuh); split across files so that they compile in parallel.
#include "survey_kernels.cuh"

namespace tp {
namespace sv {
template void launch_f<0>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<1>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<2>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<3>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<4>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<5>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<6>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<7>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
}  // namespace sv
}  // namespace tp
