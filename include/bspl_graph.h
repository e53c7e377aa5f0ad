/*
 * bspl_graph.h -- CUDA-graph capture of a batch of query calls (the paper has
 * no counterpart; the paper launches its kernels one by one from the host).
 *
 * A serving loop that runs the same query calls on the same buffers step
 * after step records them once and replays them as one graph launch:
 *
 *   bspl_graph_begin(s);                 // s: a stream other than the legacy
 *   bspl_project_curves(..., s);         //    default stream
 *   bspl_invert_curves(..., s);
 *   bspl_graph_end(s, &g, &n_kernels);   // g replays both calls
 *   for (...) bspl_graph_launch(g, s);
 *   bspl_graph_destroy(g);
 *
 * Every libbspl query entry point may be captured (they launch kernels and
 * memsets only and never synchronise); bspl_decompose, bspl_mlp_train and
 * bspl_mlp_check synchronise and must not be.  A replay reads the inputs and
 * writes the outputs at the device addresses the captured calls were given:
 * refill those buffers between replays.  Pointers are plain host handles; the
 * graph's own resources are allocated by the CUDA driver, not by libbspl.
 */
#ifndef BSPL_GRAPH_H
#define BSPL_GRAPH_H

#include <stdint.h>
#include <cuda_runtime_api.h>

#include "bspl.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef void* bspl_graph; /* an instantiated, replayable graph */

/* Starts capturing the work submitted to `stream` by this thread (thread-local
 * capture mode).  BSPL_ECUDA when the stream cannot be captured (e.g. the
 * legacy default stream, or a capture already in progress). */
bspl_status bspl_graph_begin(cudaStream_t stream);

/* Ends the capture started on `stream`, instantiates the graph and returns it
 * in *out; *n_kernels (if not NULL) receives the number of kernel launches a
 * replay makes.  BSPL_EINVAL for a NULL out, BSPL_ECUDA when capture or
 * instantiation failed (a call inside the capture did something a graph
 * cannot hold); nothing is returned then. */
bspl_status bspl_graph_end(cudaStream_t stream, bspl_graph* out, int64_t* n_kernels);

/* Replays the graph on `stream` (asynchronous).  BSPL_EINVAL for NULL. */
bspl_status bspl_graph_launch(bspl_graph g, cudaStream_t stream);

/* Releases the graph (after its last replay has finished, or with a replay
 * still queued: CUDA keeps it alive until then).  NULL is ignored. */
void bspl_graph_destroy(bspl_graph g);

#ifdef __cplusplus
}
#endif
#endif
