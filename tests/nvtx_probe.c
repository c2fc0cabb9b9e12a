/*
 * nvtx_probe.c -- a minimal NVTX tool library for the tests (test
 * infrastructure, not part of the library). The NVTX headers compiled into
 * libnpm_gb300 load it through NVTX_INJECTION64_PATH on the first range;
 * it replaces the core module's RangePushA and RangePop entries and writes
 * the name of every range pushed to the file named by NPM_NVTX_PROBE_OUT,
 * one per line.
 */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE* g_out;

static int NVTX_API probe_push(const char* name) {
    if (g_out && name) {
        fprintf(g_out, "%s\n", name);
        fflush(g_out);
    }
    return 0;
}

static int NVTX_API probe_pop(void) { return 0; }

int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size) || !table) return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)probe_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)probe_pop;
    const char* path = getenv("NPM_NVTX_PROBE_OUT");
    g_out = path ? fopen(path, "w") : NULL;
    return 1;
}
