"""Numbers the parity tests report (error over the bar, ENO2 stencil-choice
flips, the oracle's own sensitivity); the test session prints them in its
summary, so they appear in the output of a passing run too."""
NOTES = []


def note(test: str, text: str) -> None:
    NOTES.append((test, text))
