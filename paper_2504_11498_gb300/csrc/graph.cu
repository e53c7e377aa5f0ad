// CUDA-graph capture of query calls (include/bspl_graph.h): one replayable
// graph per serving step instead of one host launch per kernel.
#include "../../include/bspl_graph.h"

extern "C" {

bspl_status bspl_graph_begin(cudaStream_t stream)
{
    (void)cudaGetLastError();  // an error left over from an earlier call is not this capture's
    return cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

bspl_status bspl_graph_end(cudaStream_t stream, bspl_graph* out, int64_t* n_kernels)
{
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(stream, &graph);
    if (!out) {
        if (graph) cudaGraphDestroy(graph);
        return BSPL_EINVAL;
    }
    *out = nullptr;
    if (e != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return BSPL_ECUDA;
    }
    if (n_kernels) {
        size_t n = 0;
        int64_t k = 0;
        if (cudaGraphGetNodes(graph, nullptr, &n) == cudaSuccess && n > 0) {
            cudaGraphNode_t* nodes = new cudaGraphNode_t[n];
            if (cudaGraphGetNodes(graph, nodes, &n) == cudaSuccess)
                for (size_t i = 0; i < n; ++i) {
                    cudaGraphNodeType t;
                    if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
                }
            delete[] nodes;
        }
        *n_kernels = k;
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess || !exec) {
        cudaGetLastError();
        return BSPL_ECUDA;
    }
    *out = (bspl_graph)exec;
    return BSPL_OK;
}

bspl_status bspl_graph_launch(bspl_graph g, cudaStream_t stream)
{
    if (!g) return BSPL_EINVAL;
    return cudaGraphLaunch((cudaGraphExec_t)g, stream) == cudaSuccess ? BSPL_OK : BSPL_ECUDA;
}

void bspl_graph_destroy(bspl_graph g)
{
    if (g && cudaGraphExecDestroy((cudaGraphExec_t)g) != cudaSuccess) (void)cudaGetLastError();
}

}  // extern "C"
