"""bench.py's side legs (end to end, CPU baseline, FP64 arm, other storage,
SSOR, Table 1, serving): one that raises is reported in the line in place of
its result, and the timed solve's line is still printed."""
import bench


def test_leg_error_reports_the_exception(capsys):
    rec = bench.leg_error("ssor", RuntimeError("solve failed: status -6"))
    assert rec == {"error": "RuntimeError: solve failed: status -6"}
    assert "the ssor leg failed: RuntimeError: solve failed: status -6" in capsys.readouterr().err


def test_every_side_leg_is_guarded():
    """Each side leg's result variable is assigned by leg_error in its except
    clause (the timed region itself is not guarded: a failure there fails the
    run)."""
    import ast
    import inspect

    tree = ast.parse(inspect.getsource(bench.main))
    guarded = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Try):
            for h in node.handlers:
                for stmt in ast.walk(h):
                    if (isinstance(stmt, ast.Assign) and isinstance(stmt.value, ast.Call)
                            and getattr(stmt.value.func, "id", None) == "leg_error"):
                        guarded.add(stmt.targets[0].id)
    assert guarded == {"e2e", "cpu", "fp64_arm", "alt", "ssor", "table1", "serving"}
