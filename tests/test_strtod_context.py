"""The strtod timing context of the CPU baseline: it converts every field
(its count agrees with the oracle's for every thread split), builds with gcc
on the host, and needs no GPU."""
import pytest

import oracle
from oracle import context
from paper_2101_11408_gb300 import workloads


@pytest.mark.parametrize("threads", [1, 3, 16])
def test_field_counts_match_the_oracle(threads):
    for text, delim in ((workloads.bulk_mixed_text(20000, 91), b"\n"),
                        (workloads.uniform_text(5000), b"\n"),
                        (b"1,2\n3,,4\n\n5", b","), (b"", b"\n"), (b"7", b"\n"), (b"1\n", b"\n")):
        n, sec = context.strtod_buffer(text, delim, threads)
        bits, _ = oracle.parse_buffer(text, delim)
        assert n == bits.size, (text[:40], threads)
        assert sec >= 0.0
