// survey_inst_4.cu -- instantiations of the survey launch for several windows at once
// (feature sets 33..47 with timestamps; survey_kernels.cuh).
#include "survey_kernels.cuh"

namespace tp {
namespace sv {
template void launch_f<33>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<35>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<37>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<39>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<41>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<43>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<45>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<47>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
}  // namespace sv
}  // namespace tp
