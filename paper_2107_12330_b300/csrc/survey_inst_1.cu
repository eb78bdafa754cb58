// survey_inst_1.cu -- instantiations of the survey launch for feature sets 8..15
// (survey_kernels.cuh); split across files so that they compile in parallel.
#include "survey_kernels.cuh"

namespace tp {
namespace sv {
template void launch_f<8>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<9>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<10>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<11>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<12>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<13>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<14>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<15>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
}  // namespace sv
}  // namespace tp
