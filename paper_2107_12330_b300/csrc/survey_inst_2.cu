// survey_inst_2.cu -- instantiations of the survey launch for feature sets 16..23
// (survey_kernels.cuh); split across files so that they compile in parallel.
#include "survey_kernels.cuh"

namespace tp {
namespace sv {
template void launch_f<16>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<17>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<18>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<19>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<20>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<21>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<22>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
template void launch_f<23>(const ItemLists&, const GraphDev&, const SurveyArgs&, cudaStream_t, int, cudaEvent_t*);
}  // namespace sv
}  // namespace tp
