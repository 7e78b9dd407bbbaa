"""Every kernel launched as a programmatic dependent waits before it reads.

A kernel launched with the programmatic-stream-serialization attribute may
start while the kernel before it on the stream is still running; only its
griddepcontrol.wait (pdl_wait) orders it after that kernel.  This check reads
the CUDA sources (no GPU): for every launch that sets the attribute -- the
`pdl` flag of launch_config, or the attribute written out by a launcher --
each kernel the launch can start must execute the wait, and do so before any
statement of its body that touches global memory through its pointer
arguments.  A new kernel put on that path without the wait fails here.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_1502_02389_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = fh.read()
    return out


def _block(text, open_at):
    """The text of the brace block that opens at index open_at."""
    depth = 0
    for i in range(open_at, len(text)):
        if text[i] == "{":
            depth += 1
        elif text[i] == "}":
            depth -= 1
            if depth == 0:
                return text[open_at:i + 1]
    raise AssertionError("unbalanced braces")


def _kernel_bodies(src):
    """name -> body of every __global__ function in the sources."""
    bodies = {}
    for text in src.values():
        for m in re.finditer(r"__global__", text):
            brace = text.index("{", m.end())
            sig = re.sub(r"__launch_bounds__\s*\([^)]*\)", "", text[m.end():brace])
            name = re.search(r"(\w+)\s*\(", sig).group(1)
            bodies.setdefault(name, []).append(_block(text, brace))
    return bodies


def _pdl_launched_kernels(src):
    """Kernel names started by a launch that sets the dependent-launch attribute."""
    names = set()
    for fname, text in src.items():
        # launch_config(..., true): the kernel() of the enclosing launcher struct
        for m in re.finditer(r"launch_config\(kernel\(\),[^;]*?,\s*true\)\s*;", text, re.S):
            k = text.rfind("static const void* kernel()", 0, m.start())
            assert k >= 0, (fname, m.group(0))
            body = _block(text, text.index("{", k))
            found = re.findall(r"&(\w+)\s*<", body)
            assert found, (fname, body)
            names.update(found)
        # launchers that write the attribute out themselves
        for m in re.finditer(r"cudaLaunchAttributeProgrammaticStreamSerialization", text):
            start = text.rfind("\n}", 0, m.start())
            end = text.find("\n}", m.start())
            seg = text[start:end]
            if "lift_status launch_config(" in seg:
                continue                   # the helper itself: its callers are covered above
            found = re.findall(r"&(\w+)(?:\s*<[^>]*>)?\s*\)", seg)
            assert found, (fname, seg[-400:])
            names.update(found)
    return names


def test_every_dependent_launch_waits_before_reading():
    src = _sources()
    bodies = _kernel_bodies(src)
    names = _pdl_launched_kernels(src)
    # the families the cross-call dependent launch covers, and the second passes
    for k in ("reduce_ldg", "reduce_tma", "combine_kernel", "scal_ldg", "scal_tma", "axpy_ldg",
              "gemv_warp", "gemv_tma", "gemv_t_kernel", "gemv_t_staged", "gemv_t_combine",
              "mixed_reduce", "comp_reduce", "bs_map"):
        assert k in names, k
    for k in sorted(names):
        assert k in bodies, k
        for body in bodies[k]:
            wait = body.find("pdl_wait()")
            assert wait >= 0, f"{k} is launched as a programmatic dependent but never waits"
            # nothing before the wait dereferences memory: no indexing, no loads or stores
            head = body[:wait]
            for pat in (r"\w\s*\[[^\]]*\]\s*=(?!=)", r"ld_stream|ld_guarded|__ldg|__ldcg|bulk_g2s",
                        r"st_stream|atomicAdd|\*\s*result\s*="):
                hits = [h for h in re.findall(pat, head)
                        if not re.search(r"__shared__|mbar_init", h)]
                assert not hits, (k, pat, hits)


def test_launch_config_sets_the_attribute_only_when_asked():
    text = _sources()["api.cu"]
    k = text.index("lift_status launch_config(")
    body = _block(text, text.index("{", k))
    assert "if (pdl)" in body
    assert body.count("cudaLaunchAttributeProgrammaticStreamSerialization") == 1
