// Registry of every compiled pass kernel, gathered from the instantiation units.
#include "fftc_internal.h"

namespace fftc {

extern const KernelEntry kRowsIlTable[], kRowsSplitTable[], kColsTable[], kRowsTTable[], kTcRowsM1Table[],
    kTcRowsM2Table[], kTcRowsM3Table[], kTcRowsM4Table[], kTc4M1Table[], kTc4M2Table[], kTc4M3Table[], kTc4M4Table[], kPipeRowsIlTable[], kPipeRowsSplitTable[], kPipe4Table[], kPipeEarlyIlTable[], kPipeEarlySplitTable[],
    kColsSplitTable[], kLargeTable[], kPipeLargeTable[];
extern const int kRowsIlCount, kRowsSplitCount, kColsCount, kRowsTCount, kTcRowsM1Count, kTcRowsM2Count, kTcRowsM3Count,
    kTcRowsM4Count, kTc4M1Count, kTc4M2Count, kTc4M3Count, kTc4M4Count,
    kPipeRowsIlCount, kPipeRowsSplitCount, kPipe4Count, kPipeEarlyIlCount, kPipeEarlySplitCount, kColsSplitCount, kLargeCount, kPipeLargeCount;

struct TableRef {
    const KernelEntry *t;
    const int *n;
};
static const TableRef kTables[] = {
    {kRowsIlTable, &kRowsIlCount}, {kRowsSplitTable, &kRowsSplitCount},
    {kColsTable, &kColsCount}, {kRowsTTable, &kRowsTCount},
    {kTcRowsM1Table, &kTcRowsM1Count}, {kTcRowsM2Table, &kTcRowsM2Count},
    {kTcRowsM3Table, &kTcRowsM3Count}, {kTcRowsM4Table, &kTcRowsM4Count}, {kTc4M1Table, &kTc4M1Count},
    {kTc4M2Table, &kTc4M2Count}, {kTc4M3Table, &kTc4M3Count}, {kTc4M4Table, &kTc4M4Count},
    {kPipeRowsIlTable, &kPipeRowsIlCount}, {kPipeRowsSplitTable, &kPipeRowsSplitCount}, {kPipe4Table, &kPipe4Count},
    {kPipeEarlyIlTable, &kPipeEarlyIlCount}, {kPipeEarlySplitTable, &kPipeEarlySplitCount},
    {kColsSplitTable, &kColsSplitCount}, {kLargeTable, &kLargeCount},
    {kPipeLargeTable, &kPipeLargeCount},
};

int kernel_count() {
    int c = 0;
    for (const TableRef &r : kTables) c += *r.n;
    return c;
}

const KernelEntry *kernel_at(int i) {
    if (i < 0) return nullptr;
    for (const TableRef &r : kTables) {
        if (i < *r.n) return &r.t[i];
        i -= *r.n;
    }
    return nullptr;
}

}  // namespace fftc
