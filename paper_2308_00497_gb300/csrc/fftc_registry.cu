// Registry of every compiled pass kernel, gathered from the instantiation units.
#include "fftc_internal.h"

namespace fftc {

extern const KernelEntry kRowsIlTable[], kRowsSplitTable[], kColsTable[], kRowsTTable[], kTcRowsTable[],
    kTc4Table[], kPipeRowsIlTable[], kPipeRowsSplitTable[], kPipe4Table[], kPipeEarlyIlTable[], kPipeEarlySplitTable[],
    kColsSplitTable[], kLargeTable[], kPipeLargeTable[];
extern const int kRowsIlCount, kRowsSplitCount, kColsCount, kRowsTCount, kTcRowsCount, kTc4Count,
    kPipeRowsIlCount, kPipeRowsSplitCount, kPipe4Count, kPipeEarlyIlCount, kPipeEarlySplitCount, kColsSplitCount, kLargeCount, kPipeLargeCount;

struct TableRef {
    const KernelEntry *t;
    const int *n;
};
static const TableRef kTables[] = {
    {kRowsIlTable, &kRowsIlCount}, {kRowsSplitTable, &kRowsSplitCount},
    {kColsTable, &kColsCount}, {kRowsTTable, &kRowsTCount},
    {kTcRowsTable, &kTcRowsCount}, {kTc4Table, &kTc4Count},
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
