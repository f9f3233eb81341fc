"""Plain FP64 CPU oracle for the QR-based CT reconstruction path (test
infrastructure only; see ``oracle.py``)."""
