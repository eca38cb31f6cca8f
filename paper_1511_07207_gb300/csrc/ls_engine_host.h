// ls_engine_host.h -- host-side engine object shared by ls_batch_solve and the
// server.
#pragma once

#include <vector>

#include "ls_api_internal.h"
#include "ls_engine.h"

namespace lsi {

struct SlotResult {
    int status, inner, outer, done;
    double rel_res;                 // worst column
    double colres[E_MAXS];          // ||R_j|| / ||B_j|| per column
};

// Copy of columns [c0, c0 + k) of a slot's X to a column-major destination.
struct FinishItem {
    int slot, c0, k;
    double *x;
    long long ldx;
};

// Tile shape of a slot's FP32 products (ls_tune.cu): columns of A per task and
// whether the products run on the tensor cores.
struct TuneChoice {
    int ks32;
    int tc;
};
TuneChoice tune_choice(const ls_ctx *c, int n, int s);

struct SlotSizes {
    int sp;
    int ks32, tc;        // tuned tile shape
    long long ld32, lda_stage;
    size_t bytes;        // engine buffers of the slot
    size_t stageA;       // FP64 copy of a host A
    size_t stageBX;      // column-major copy of a host B or X
};

SlotSizes slot_sizes(const ls_ctx *c, int n, int s, int method, int m);
void slot_carve(SlotDesc &D, const SlotSizes &z, char *base, int n, int s, int method, int m);

class Engine {
public:
    ls_ctx *c = nullptr;
    int cap_slots = 0, cap32 = 0, capb = 0, cap64 = 0, capv = 0;
    int nb32 = 0;                        // FP32 row blocks in the current tables
    char *dmem = nullptr;
    size_t dbytes = 0;
    EngineDev *dE = nullptr;
    EngineDev hE{};
    const double **bsrc = nullptr;
    long long *ldb = nullptr;
    double **xdst = nullptr;           // finish items (capacity cap_slots * E_MAXS)
    long long *ldx = nullptr;
    int *fslot = nullptr, *fc0 = nullptr, *fk = nullptr;
    SlotResult *results = nullptr;
    std::vector<Task> h32, h64, hv;
    std::vector<int> h_order;            // eng_red block -> slot (costliest first)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    EngineKernels K{};
    int grid_prod = 0, grid_vec = 0;

    ~Engine();
    void release();
    int reserve(ls_ctx *ctx, int slots, int n32, int nrb, int n64, int nv);
    int build_graph();
    void set_tasks(std::vector<SlotDesc> &hd, int fixed_max_n);
    int upload(const std::vector<SlotDesc> &hd, int tick_limit, bool tables);
    int init_slots(int first, int count);
    int admit(int first, int count, const std::vector<const double *> &bs,
              const std::vector<long long> &lb);
    int finish(const std::vector<FinishItem> &items);
    int collect(int first, int count, std::vector<SlotResult> &out);
    int run();
    unsigned long long launches();
};

}  // namespace lsi
