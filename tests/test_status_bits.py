"""The status bits of include/wfpg.h and the binding's constants agree (host
only: the header is read as text)."""
import os
import re

from paper_2405_06997_gb300 import wfpg as W

HEADER = os.path.join(os.path.dirname(__file__), "..", "include", "wfpg.h")


def header_status_bits():
    text = open(HEADER).read()
    return {m.group(1): 1 << int(m.group(2)) for m in re.finditer(r"WFPG_STATUS_(\w+)\s*=\s*1u\s*<<\s*(\d+)", text)}


def test_status_bits_match_the_binding():
    bits = header_status_bits()
    assert set(bits) == {"TRACE_CAP", "BIN_CAPACITY", "RUN_SIZES", "MMA_TIMEOUT", "WAIT_TIMEOUT"}
    for name, value in bits.items():
        assert getattr(W, "STATUS_" + name) == value, name
    assert len(set(bits.values())) == len(bits)  # distinct bits
