/* A minimal NVTX injection library for the tests: when NVTX_INJECTION64_PATH
 * names it, every range pushed and popped through NVTX is written as a line
 * ("push <name>" / "pop") to the file NVTX_RECORD_PATH names. It uses only the
 * public injection interface of the NVTX v3 headers. */
#include <nvtx3/nvToolsExt.h>

#include <stdio.h>
#include <stdlib.h>

static FILE* g_out;

static int NVTX_API record_push(const char* name) {
    if (g_out) { fprintf(g_out, "push %s\n", name ? name : ""); fflush(g_out); }
    return 0;
}

static int NVTX_API record_pop(void) {
    if (g_out) { fputs("pop\n", g_out); fflush(g_out); }
    return 0;
}

int NVTX_API InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table) {
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int last = 0;
    if (!cb || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &last)) return 0;
    if (last < NVTX_CBID_CORE_RangePop) return 0;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    const char* path = getenv("NVTX_RECORD_PATH");
    g_out = path ? fopen(path, "w") : NULL;
    return 1;
}
