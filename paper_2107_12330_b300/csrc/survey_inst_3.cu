// survey_inst_3.cu -- instantiations of the survey launch for feature sets 24..31
// (survey_kernels.cuh); split across files so that they compile in parallel.
#include "survey_kernels.cuh"

namespace tp {
namespace sv {
template void launch_f<24>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<25>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<26>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<27>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<28>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<29>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<30>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<31>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
}  // namespace sv
}  // namespace tp
