"""Stored expected values: ones the paper prints (cited) and ones written by the
scripts here, which call only the oracle and the seeded input generators."""
