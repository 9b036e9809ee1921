"""Every device buffer the context owns is released by afd_destroy: the
release list in the ABI implementation names each DevBuf member of the
context struct (a buffer added to the context but not to the list would
leak device memory at every destroy). Source check, no GPU needed."""
import os
import re

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1907_02290_gb300", "csrc")


def test_destroy_releases_every_context_buffer():
    h = open(os.path.join(CSRC, "afd_internal.cuh")).read()
    a = h.index("struct afd_ctx")
    body = h[a:h.index("\n};", a)]
    members = []
    for line in body.split("\n"):
        m = re.match(r"\s*afd::DevBuf\s+(.*);", line.split("//")[0])
        if m:
            members += [x.strip() for x in m.group(1).split(",")]
    api = open(os.path.join(CSRC, "afd_api.cu")).read()
    d = api.index("void afd_destroy")
    released = set(re.findall(r"&c->(\w+)", api[d:api.index("for (DevBuf *b : bufs)", d)]))
    assert len(members) > 100
    assert [m for m in members if m not in released] == []
