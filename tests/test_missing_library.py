"""Without liblb.so the binding fails loudly: every call raises ImportError,
and nothing is computed on the CPU instead (there is no fallback path)."""
import os
import subprocess
import sys
import textwrap

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_call_raises_when_the_library_is_absent():
    absent = os.path.join(ROOT, "_build", "absent", "liblb.so")
    assert not os.path.exists(absent)
    code = textwrap.dedent("""
        import sys
        sys.path.insert(0, %r)
        from paper_1310_4218_gb300 import lb
        lb.LIB_PATH = %r
        calls = {
            "lb_default_options": lambda: lb.lb_default_options(),
            "lb_plan": lambda: lb.lb_plan("greedy", [1.0, 2.0, 3.0], 2),
            "lb_create": lambda: lb.lb_create([], [(0, 0, 0, 1, 1)]),
        }
        for name, call in calls.items():
            try:
                call()
            except ImportError as e:
                assert "not built" in str(e), (name, str(e))
            else:
                raise SystemExit(name + " returned without the library")
        print("ok")
    """) % (ROOT, absent)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip() == "ok"
